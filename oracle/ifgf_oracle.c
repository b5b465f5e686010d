/*
 * CPU FP64 oracle for the Interpolated Factored Green Function (IFGF) method of
 * Bauinger & Bruno, arXiv 2010.02857.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled and called by the test
 * suite, by the package's smoke check and by the benchmark's CPU-baseline leg.
 * The GPU library never links, loads or calls it, and it shares no code with
 * the GPU library.
 *
 * It is a plain, slow, serial-order implementation written for reading against
 * the paper:
 *   - oracle_direct / oracle_direct_adjoint: the exact discrete operator of
 *     Eq. (field1) with the Helmholtz kernel of Eq. (greensfunction), and its
 *     conjugate transpose, by a double loop (self term skipped, Eq. field1).
 *   - oracle_plan_* / oracle_apply: Algorithm 1 ("IFGF Method", Sec. 3.3.3) with
 *     the box octree, cousins and relevant cone segments of Sec. 3.3.1, the
 *     factorization of Eq. (factor)/(factored_f), the s change of variables of
 *     Eq. (defparametrizationins)/(def_eps), the cone domains of
 *     Eq. (defconedomain)/(defconedomainproduct) and the Chebyshev interpolation
 *     of Eq. (defchebyshevinterpooperator) evaluated in Lagrange form at the
 *     first-kind nodes x_k = cos((2k+1)pi/(2n)).
 *   - oracle_apply_adjoint: the exact transpose of every linear step of
 *     Algorithm 1, in reverse order (the paper has no adjoint; this is linear
 *     algebra on the same steps).
 *
 * Readings of passages that the paper leaves open (all exercised by tests):
 *   R1  g_S carries no 1/(4 pi): G(x,x_S) g_S(x,x') = G(x,x') (Eq. factored_f).
 *   R2  Interpolation is the unique polynomial through the first-kind
 *       Chebyshev nodes (Eq. defchebyshevinterpooperator), in Lagrange form;
 *       the printed coefficient formula (Eq. defchebyshevcoeffsandpoints) mixes
 *       endpoint weights and is not used.
 *   R3  P_s and P_ang count points per axis: P = P_s * P_ang^2 nodes per cone.
 *   R4  Cone cells are half-open; cell indices come from comparisons of
 *       v_z/r and v_x/rho with cos(k pi / n_C), never from inverse trig;
 *       on the axis (rho == 0) the paper's pole rule of Eq. (defconedomain)
 *       is used (theta = 0 -> first phi cell, theta = pi -> last phi cell).
 *   R5  Refinement multiplies: n_{.,d-1} = a_d n_{.,d}, a_d = 2 iff
 *       2 kappa H_d > 1, else 1 (Sec. 3.3.1, cone hierarchy paragraph).
 *   R6  Root box: the bounding cube of the points, side = largest extent,
 *       centred at the bounding-box midpoint; integer box coordinates are
 *       clamped to [0, 2^{d-1} - 1] (the half-open box of Eq. defbox excludes
 *       the upper face).
 *   R7  Relevance rule (ii) uses the parent cones' interpolation points
 *       (Sec. 3.3.2, first paragraph), not whole-segment overlap.
 *   R8  D counts the root as level 1; cones exist at levels 3..D; the upward
 *       step runs only for d > 3 (Algorithm 1).
 *   R9  A parent cone's interpolation point seen from a child centre is
 *       evaluated as R dir - delta, delta = (+-H_d/2)^3 (Eq. interp_pts with
 *       Eq. defboxsizesandcenters), not as the difference of two rounded
 *       absolute positions; the result is independent of the boxes' location.
 *
 * Floating-point contract for the index path (box and cone indices): only the
 * correctly rounded operations + - * / sqrt are used, in the order written, and
 * the file must be compiled with -ffp-contract=off so that no fused
 * multiply-add changes a rounding.  Trigonometric values that feed indices or
 * node positions come from tables computed once per level with libm.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORACLE_MAXLEV 22

/* ------------------------------------------------------------------------- */
/* Kernel of Eq. (greensfunction) and analytic factor of Eq. (factored_f).    */
/* ------------------------------------------------------------------------- */

static double dist3(const double *x, const double *y)
{
    double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* G(x, y) = exp(i kappa |x - y|) / (4 pi |x - y|) */
static cplx green(const double *x, const double *y, double kappa)
{
    double r = dist3(x, y);
    return cexp(I * kappa * r) / (4.0 * M_PI * r);
}

/* g_S(x, x') = |x - x_S| / |x - x'| * exp(i kappa (|x - x'| - |x - x_S|)) */
static cplx analytic_factor(const double *x, const double *xs, const double *xp, double kappa)
{
    double r0 = dist3(x, xs);
    double r1 = dist3(x, xp);
    return (r0 / r1) * cexp(I * kappa * (r1 - r0));
}

void oracle_green(const double *x, const double *y, double kappa, double *out)
{
    cplx g = green(x, y, kappa);
    out[0] = creal(g);
    out[1] = cimag(g);
}

void oracle_analytic_factor(const double *x, const double *xs, const double *xp, double kappa,
                            double *out)
{
    cplx g = analytic_factor(x, xs, xp, kappa);
    out[0] = creal(g);
    out[1] = cimag(g);
}

/* ------------------------------------------------------------------------- */
/* Direct evaluation of Eq. (field1): I(x_l) = sum_{m != l} a_m G(x_l, x_m).  */
/* a: [nrhs][n] complex; out: [nrhs][m] complex at the listed targets.        */
/* ------------------------------------------------------------------------- */
void oracle_direct(int64_t n, const double *pts, double kappa, int nrhs, const double *a_in,
                   int64_t m, const int64_t *targets, double *out_)
{
    const cplx *a = (const cplx *)a_in;
    cplx *out = (cplx *)out_;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < m; ++t) {
        int64_t l = targets[t];
        cplx acc[nrhs];
        for (int r = 0; r < nrhs; ++r) acc[r] = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == l) continue;
            cplx g = green(pts + 3 * l, pts + 3 * j, kappa);
            for (int r = 0; r < nrhs; ++r) acc[r] += a[(int64_t)r * n + j] * g;
        }
        for (int r = 0; r < nrhs; ++r) out[(int64_t)r * m + t] = acc[r];
    }
}

/* Conjugate transpose of Eq. (field1): (A^H v)_m = sum_{l != m} conj(G(x_l, x_m)) v_l,
 * evaluated at the listed source indices. */
void oracle_direct_adjoint(int64_t n, const double *pts, double kappa, int nrhs, const double *v_in,
                           int64_t m, const int64_t *sources, double *out_)
{
    const cplx *v = (const cplx *)v_in;
    cplx *out = (cplx *)out_;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < m; ++t) {
        int64_t s = sources[t];
        cplx acc[nrhs];
        for (int r = 0; r < nrhs; ++r) acc[r] = 0;
        for (int64_t l = 0; l < n; ++l) {
            if (l == s) continue;
            cplx g = conj(green(pts + 3 * l, pts + 3 * s, kappa));
            for (int r = 0; r < nrhs; ++r) acc[r] += v[(int64_t)r * n + l] * g;
        }
        for (int r = 0; r < nrhs; ++r) out[(int64_t)r * m + t] = acc[r];
    }
}

/* ------------------------------------------------------------------------- */
/* 1-D Chebyshev interpolation (Eq. defchebyshevinterpooperator), reading R2. */
/* ------------------------------------------------------------------------- */

/* first-kind Chebyshev nodes x_k = cos((2k+1) pi / (2n)), k = 0..n-1 */
static void cheb_nodes(int n, double *t)
{
    for (int k = 0; k < n; ++k) t[k] = cos(((double)(2 * k + 1) * M_PI) / (double)(2 * n));
}

/* Lagrange basis at the nodes: L_a(t) = prod_{e != a} (t - t_e) / (t_a - t_e) */
static void lagrange(int n, const double *nodes, double t, double *w)
{
    for (int a = 0; a < n; ++a) {
        double v = 1.0;
        for (int e = 0; e < n; ++e)
            if (e != a) v *= (t - nodes[e]) / (nodes[a] - nodes[e]);
        w[a] = v;
    }
}

void oracle_cheb_nodes(int n, double *t) { cheb_nodes(n, t); }

void oracle_lagrange(int n, double t, double *w)
{
    double nodes[64];
    cheb_nodes(n, nodes);
    lagrange(n, nodes, t, w);
}

/* ------------------------------------------------------------------------- */
/* Plan: box octree (Sec. 3.3.1), cousins (Eq. defcousinboxes), cone levels   */
/* and relevant cone segments (Eq. defallrelevantconesegments, reading R7).   */
/* ------------------------------------------------------------------------- */

typedef struct {
    /* boxes of one level, in ascending Morton order */
    int64_t nbox;
    uint64_t *key;     /* Morton key of the box's integer coordinate */
    int64_t *start;    /* [nbox+1] first sorted point of the box (start[nbox] = n) */
    int64_t *end;      /* [nbox] one past its last point: start[b+1] in a uniform tree; in
                        * an adaptive tree the points of coarser leaves lie between boxes */
    unsigned char *leaf; /* [nbox] the box is a leaf (not subdivided) */
    int64_t *near_start, *near_lo, *near_hi; /* leaf boxes: CSR of the point ranges of
                        * the near field of their targets, ascending (reading R13) */
    int64_t *parent;   /* index of the parent box at level d-1 (level >= 2) */
    int64_t *child0;   /* [nbox+1] first child at level d+1 (level < D) */
    int64_t *nbr_start, *nbr;   /* neighbours N B (includes the box itself) */
    int64_t *cous_start, *cous; /* cousins M B (level >= 3) */
    /* cone level (levels >= 3) */
    int ns, nc;
    double H, h, ds, dth;
    double *cosk;      /* [nc+1] cos(k pi / nc) */
    double *nodeR;     /* [ns*Ps] h / s_a */
    double *sth, *cth; /* [nc*Pang] sin / cos of theta nodes */
    double *sph, *cph; /* [2nc*Pang] sin / cos of phi nodes */
    /* relevant cones */
    int64_t *act_start; /* [nbox+1] */
    int64_t *act_cone;  /* sorted cone ids per box */
    int64_t nact;
    cplx *F;            /* [nact][P][nrhs] after an apply */
    cplx *Fadj;         /* adjoint accumulators */
    int64_t cousin_evals, upward_evals;
} olevel;

typedef struct {
    int64_t n;
    int D, Ps, Pang, P;
    double kappa;
    double H1, corner[3];
    int64_t *perm;   /* sorted position -> user index */
    double *xs;      /* sorted points [n][3] */
    uint64_t *leafkey;
    int64_t leaf_max; /* adaptive tree: a box with at most leaf_max points is a leaf (0: uniform) */
    int *ptlev;      /* [n] level of the leaf box of each sorted point */
    double ts[64], ta[64]; /* Chebyshev nodes for P_s and P_ang */
    olevel lev[ORACLE_MAXLEV + 1];
    int nrhs_F;
    int64_t near_pairs;
    int err;
} oplan;

static uint64_t morton3(uint64_t kx, uint64_t ky, uint64_t kz)
{
    uint64_t key = 0;
    for (int b = 0; b < 21; ++b) {
        key |= ((kx >> b) & 1ull) << (3 * b);
        key |= ((ky >> b) & 1ull) << (3 * b + 1);
        key |= ((kz >> b) & 1ull) << (3 * b + 2);
    }
    return key;
}

static void demorton3(uint64_t key, int64_t *k)
{
    k[0] = k[1] = k[2] = 0;
    for (int b = 0; b < 21; ++b) {
        k[0] |= (int64_t)((key >> (3 * b)) & 1ull) << b;
        k[1] |= (int64_t)((key >> (3 * b + 1)) & 1ull) << b;
        k[2] |= (int64_t)((key >> (3 * b + 2)) & 1ull) << b;
    }
}

typedef struct { uint64_t key; int64_t idx; } keyidx;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y);
}

/* index of `key` in the sorted array, or -1 */
static int64_t find_key(const uint64_t *keys, int64_t n, uint64_t key)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (keys[mid] < key) lo = mid + 1; else hi = mid;
    }
    return (lo < n && keys[lo] == key) ? lo : -1;
}

static int64_t find_i64(const int64_t *v, int64_t lo, int64_t hi, int64_t x)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (v[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* centre of box with integer coordinate k at level d, Eq. (defboxsizesandcenters):
 * x_k^d = corner + (k + 1/2) H_d, with 0-based k. */
static void box_center(const oplan *p, int d, uint64_t key, double *c)
{
    int64_t k[3];
    demorton3(key, k);
    double H = p->lev[d].H;
    for (int i = 0; i < 3; ++i) c[i] = p->corner[i] + ((double)k[i] + 0.5) * H;
}

/* Cone cell of point y relative to centre c at level d (reading R4).  Returns the
 * linear id (g1 * nc + g2) * 2nc + g3 and, if loc != NULL, the local coordinates
 * in [-1, 1] of (s, theta, phi) within the cell. */
static int64_t cone_of_vec(const oplan *p, int d, const double *v, int64_t *g, double *loc)
{
    const olevel *L = &p->lev[d];
    double vx = v[0], vy = v[1], vz = v[2];
    double rho2 = vx * vx + vy * vy;
    double r = sqrt(rho2 + vz * vz);
    double rho = sqrt(rho2);
    int nc = L->nc, ns = L->ns;
    int64_t g1, g2, g3;
    if (r == 0.0) {
        g1 = g2 = g3 = 0;
    } else {
        double s = L->h / r;
        double q = floor(s / L->ds);
        g1 = q < 0 ? 0 : (q > ns - 1 ? ns - 1 : (int64_t)q);
        double ct = vz / r;
        g2 = 0;
        for (int k = 1; k <= nc - 1; ++k)
            if (ct <= L->cosk[k]) g2++;
        if (rho == 0.0) {
            g3 = vz > 0.0 ? 0 : 2 * nc - 1;
        } else {
            double cp = vx / rho;
            if (vy >= 0.0) {
                g3 = 0;
                for (int j = 1; j <= nc; ++j)
                    if (cp <= L->cosk[j]) g3++;
            } else {
                g3 = nc;
                for (int j = 1; j <= nc - 1; ++j)
                    if (cp >= -L->cosk[j]) g3++;
            }
        }
        if (loc) {
            loc[0] = 2.0 * (s / L->ds - (double)g1) - 1.0;
            double th = atan2(rho, vz);
            loc[1] = 2.0 * (th / L->dth - (double)g2) - 1.0;
            if (rho == 0.0) {
                loc[2] = 0.0; /* on the axis the field does not depend on phi */
            } else {
                double ph = atan2(vy, vx);
                if (ph < 0.0) ph += 2.0 * M_PI;
                loc[2] = 2.0 * (ph / L->dth - (double)g3) - 1.0;
            }
        }
    }
    if (g) { g[0] = g1; g[1] = g2; g[2] = g3; }
    return (g1 * nc + g2) * (2 * nc) + g3;
}

/* Cone cell of point y relative to centre c at level d: the vector y - c. */
static int64_t cone_of(const oplan *p, int d, const double *y, const double *c, int64_t *g, double *loc)
{
    double v[3] = {y[0] - c[0], y[1] - c[1], y[2] - c[2]};
    return cone_of_vec(p, d, v, g, loc);
}

/* Interpolation point p = (a, b, c) of cone `cone` around centre x at level d,
 * Eq. (interp_pts): x^d(s_a, theta_b, phi_c) + x.  Returns |point - x| as the
 * table radius h_d / s_a. */
static double node_pos(const oplan *p, int d, int64_t cone, int node, const double *x, double *q)
{
    const olevel *L = &p->lev[d];
    int nc = L->nc, Pa = p->Pang;
    int64_t g3 = cone % (2 * nc);
    int64_t g2 = (cone / (2 * nc)) % nc;
    int64_t g1 = cone / (2 * nc) / nc;
    int a = node / (Pa * Pa), b = (node / Pa) % Pa, c = node % Pa;
    double R = L->nodeR[g1 * p->Ps + a];
    double st = L->sth[g2 * Pa + b], ct = L->cth[g2 * Pa + b];
    double sp = L->sph[g3 * Pa + c], cp = L->cph[g3 * Pa + c];
    q[0] = x[0] + R * (st * cp);
    q[1] = x[1] + R * (st * sp);
    q[2] = x[2] + R * ct;
    return R;
}

/* Interpolation point `node` of the level-(d-1) cone `cone` of a parent box, relative
 * to the centre of its child box with octant bits `oct` (bit 0: x, 1: y, 2: z) at
 * level d.  By Eq. (interp_pts) the point is x_j + R dir with R = h_{d-1}/s_a, and by
 * Eq. (defboxsizesandcenters) the child centre is x_j + delta with
 * delta_i = +H_d/2 (bit set) or -H_d/2, so the point relative to the child centre
 * is R dir - delta.  It is evaluated in that form, which does not depend on where
 * the boxes are.  Returns R; dir receives the unit direction. */
static double node_rel_child(const oplan *p, int d, int64_t cone, int node, int oct, double *v, double *dir)
{
    const olevel *L = &p->lev[d - 1];
    int nc = L->nc, Pa = p->Pang;
    int64_t g3 = cone % (2 * nc);
    int64_t g2 = (cone / (2 * nc)) % nc;
    int64_t g1 = cone / (2 * nc) / nc;
    int a = node / (Pa * Pa), b = (node / Pa) % Pa, c = node % Pa;
    double R = L->nodeR[g1 * p->Ps + a];
    double st = L->sth[g2 * Pa + b], ct = L->cth[g2 * Pa + b];
    double sp = L->sph[g3 * Pa + c], cp = L->cph[g3 * Pa + c];
    double hh = p->lev[d].H * 0.5;
    double dx = st * cp, dy = st * sp, dz = ct;
    v[0] = R * dx - ((oct & 1) ? hh : -hh);
    v[1] = R * dy - ((oct & 2) ? hh : -hh);
    v[2] = R * dz - ((oct & 4) ? hh : -hh);
    if (dir) { dir[0] = dx; dir[1] = dy; dir[2] = dz; }
    return R;
}

void oracle_node_rel_child(void *h, int d, int64_t cone, int node, int oct, double *v)
{
    node_rel_child(h, d, cone, node, oct, v, NULL);
}

/* slot of cone id in box b's relevant list, or -1 */
static int64_t find_slot(const olevel *L, int64_t b, int64_t cone)
{
    int64_t lo = L->act_start[b], hi = L->act_start[b + 1];
    int64_t pos = find_i64(L->act_cone, lo, hi, cone);
    return (pos < hi && L->act_cone[pos] == cone) ? pos : -1;
}

static void free_level(olevel *L)
{
    free(L->key); free(L->start); free(L->end); free(L->leaf); free(L->parent); free(L->child0);
    free(L->near_start); free(L->near_lo); free(L->near_hi);
    free(L->nbr_start); free(L->nbr); free(L->cous_start); free(L->cous);
    free(L->cosk); free(L->nodeR); free(L->sth); free(L->cth); free(L->sph); free(L->cph);
    free(L->act_start); free(L->act_cone); free(L->F); free(L->Fadj);
    memset(L, 0, sizeof(*L));
}

void oracle_plan_destroy(void *h)
{
    oplan *p = h;
    if (!p) return;
    for (int d = 0; d <= ORACLE_MAXLEV; ++d) free_level(&p->lev[d]);
    free(p->perm); free(p->xs); free(p->leafkey); free(p->ptlev);
    free(p);
}

/* dynamic int64 vector */
typedef struct { int64_t *v; int64_t n, cap; } ivec;
static void ipush(ivec *a, int64_t x)
{
    if (a->n == a->cap) {
        a->cap = a->cap ? 2 * a->cap : 64;
        a->v = realloc(a->v, (size_t)a->cap * sizeof(int64_t));
    }
    a->v[a->n++] = x;
}

/* sort + unique an int64 array in place, returns the new length */
static int64_t sort_unique(int64_t *v, int64_t n)
{
    if (n == 0) return 0;
    qsort(v, (size_t)n, sizeof(int64_t), cmp_i64);
    int64_t m = 1;
    for (int64_t i = 1; i < n; ++i)
        if (v[i] != v[m - 1]) v[m++] = v[i];
    return m;
}

static int cmp_range(const void *a, const void *b)
{
    const int64_t *x = a, *y = b;
    return x[0] < y[0] ? -1 : (x[0] > y[0]);
}

/*
 * Build the plan.  pts: [n][3] user order.  leaf_max = 0 builds the uniform octree of
 * D levels (Sec. 3.3.1); leaf_max > 0 the adaptive one of reading R13: a box of level
 * >= 3 with at most leaf_max points is not subdivided.  Returns NULL on invalid input
 * (n < 2, D < 3, D > 22, P < 1, kappa < 0, leaf_max < 0, non-finite coordinates).
 */
static void *plan_create(int64_t n, const double *pts, double kappa, int D, int Ps, int Pang,
                         int leaf_ns, int leaf_nc, int64_t leaf_max)
{
    if (n < 2 || D < 3 || D > ORACLE_MAXLEV || Ps < 1 || Pang < 1 || Ps > 64 || Pang > 64 ||
        kappa < 0 || leaf_ns < 1 || leaf_nc < 1 || leaf_max < 0)
        return NULL;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(pts[i])) return NULL;
    oplan *p = calloc(1, sizeof(oplan));
    p->n = n; p->D = D; p->Ps = Ps; p->Pang = Pang; p->P = Ps * Pang * Pang; p->kappa = kappa;
    cheb_nodes(Ps, p->ts);
    cheb_nodes(Pang, p->ta);

    /* root box (reading R6) */
    double lo[3], hi[3];
    for (int i = 0; i < 3; ++i) lo[i] = hi[i] = pts[i];
    for (int64_t j = 0; j < n; ++j)
        for (int i = 0; i < 3; ++i) {
            if (pts[3 * j + i] < lo[i]) lo[i] = pts[3 * j + i];
            if (pts[3 * j + i] > hi[i]) hi[i] = pts[3 * j + i];
        }
    double H1 = 0.0;
    for (int i = 0; i < 3; ++i)
        if (hi[i] - lo[i] > H1) H1 = hi[i] - lo[i];
    if (!(H1 > 0.0)) { free(p); return NULL; }
    p->H1 = H1;
    for (int i = 0; i < 3; ++i) p->corner[i] = (lo[i] + hi[i]) * 0.5 - H1 * 0.5;
    for (int d = 1; d <= D; ++d) p->lev[d].H = ldexp(H1, -(d - 1));

    /* leaf coordinates, Morton keys, stable sort (ties by user index) */
    double HD = p->lev[D].H;
    int64_t nside = (int64_t)1 << (D - 1);
    keyidx *ki = malloc((size_t)n * sizeof(keyidx));
    for (int64_t j = 0; j < n; ++j) {
        int64_t k[3];
        for (int i = 0; i < 3; ++i) {
            double q = floor((pts[3 * j + i] - p->corner[i]) / HD);
            k[i] = q < 0 ? 0 : (q > (double)(nside - 1) ? nside - 1 : (int64_t)q);
        }
        ki[j].key = morton3((uint64_t)k[0], (uint64_t)k[1], (uint64_t)k[2]);
        ki[j].idx = j;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    p->perm = malloc((size_t)n * sizeof(int64_t));
    p->xs = malloc((size_t)n * 3 * sizeof(double));
    p->leafkey = malloc((size_t)n * sizeof(uint64_t));
    for (int64_t j = 0; j < n; ++j) {
        p->perm[j] = ki[j].idx;
        p->leafkey[j] = ki[j].key;
        for (int i = 0; i < 3; ++i) p->xs[3 * j + i] = pts[3 * ki[j].idx + i];
    }
    free(ki);

    /* relevant boxes per level: unique level keys of the sorted points.  In the
     * adaptive tree (reading R13) a box exists when its parent exists and is not a
     * leaf; a box is a leaf at level D, or at a level >= 3 when it holds at most
     * leaf_max points.  The points of a level's boxes are contiguous per box; the
     * points of coarser leaves lie between them (start/end per box). */
    p->leaf_max = leaf_max;
    p->ptlev = malloc((size_t)n * sizeof(int));
    for (int64_t j = 0; j < n; ++j) p->ptlev[j] = D;
    for (int d = 1; d <= D; ++d) {
        olevel *L = &p->lev[d];
        int sh = 3 * (D - d);
        int64_t nb = 0;
        for (int64_t j = 0; j < n; ++j)
            if (p->ptlev[j] >= d && (j == 0 || p->ptlev[j - 1] < d || (p->leafkey[j] >> sh) != (p->leafkey[j - 1] >> sh)))
                nb++;
        L->nbox = nb;
        L->key = malloc((size_t)(nb > 0 ? nb : 1) * sizeof(uint64_t));
        L->start = malloc((size_t)(nb + 1) * sizeof(int64_t));
        L->end = malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int64_t));
        L->leaf = malloc((size_t)(nb > 0 ? nb : 1));
        int64_t b = -1;
        for (int64_t j = 0; j < n; ++j) {
            if (p->ptlev[j] < d) continue;
            if (b < 0 || p->ptlev[j - 1] < d || (p->leafkey[j] >> sh) != (p->leafkey[j - 1] >> sh)) {
                ++b;
                L->key[b] = p->leafkey[j] >> sh;
                L->start[b] = j;
            }
            L->end[b] = j + 1;
        }
        L->start[nb] = n;
        for (b = 0; b < nb; ++b) {
            L->leaf[b] = d == D || (leaf_max > 0 && d >= 3 && L->end[b] - L->start[b] <= leaf_max);
            if (L->leaf[b] && d < D)
                for (int64_t j = L->start[b]; j < L->end[b]; ++j) p->ptlev[j] = d;
        }
    }
    /* parent / children */
    for (int d = 2; d <= D; ++d) {
        olevel *L = &p->lev[d], *Lp = &p->lev[d - 1];
        L->parent = malloc((size_t)L->nbox * sizeof(int64_t));
        for (int64_t b = 0; b < L->nbox; ++b) L->parent[b] = find_key(Lp->key, Lp->nbox, L->key[b] >> 3);
        Lp->child0 = malloc((size_t)(Lp->nbox + 1) * sizeof(int64_t));
        int64_t c = 0;
        for (int64_t b = 0; b < Lp->nbox; ++b) {
            while (c < L->nbox && L->parent[c] < b) c++;
            Lp->child0[b] = c;
        }
        Lp->child0[Lp->nbox] = L->nbox;
    }
    /* neighbours: relevant boxes a with |a - k|_inf <= 1, in ascending order */
    for (int d = 1; d <= D; ++d) {
        olevel *L = &p->lev[d];
        int64_t side = (int64_t)1 << (d - 1);
        L->nbr_start = malloc((size_t)(L->nbox + 1) * sizeof(int64_t));
        ivec list = {0};
        for (int64_t b = 0; b < L->nbox; ++b) {
            L->nbr_start[b] = list.n;
            int64_t k[3];
            demorton3(L->key[b], k);
            int64_t tmp[27];
            int nt = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int64_t a0 = k[0] + dx, a1 = k[1] + dy, a2 = k[2] + dz;
                        if (a0 < 0 || a1 < 0 || a2 < 0 || a0 >= side || a1 >= side || a2 >= side) continue;
                        int64_t f = find_key(L->key, L->nbox, morton3(a0, a1, a2));
                        if (f >= 0) tmp[nt++] = f;
                    }
            qsort(tmp, (size_t)nt, sizeof(int64_t), cmp_i64);
            for (int i = 0; i < nt; ++i) ipush(&list, tmp[i]);
        }
        L->nbr_start[L->nbox] = list.n;
        L->nbr = list.v;
    }
    /* cousins, Eq. (defcousinboxes): children of the parent's neighbours that are
     * not neighbours of the box; ascending order */
    for (int d = 3; d <= D; ++d) {
        olevel *L = &p->lev[d], *Lp = &p->lev[d - 1];
        L->cous_start = malloc((size_t)(L->nbox + 1) * sizeof(int64_t));
        ivec list = {0};
        for (int64_t b = 0; b < L->nbox; ++b) {
            L->cous_start[b] = list.n;
            int64_t k[3];
            demorton3(L->key[b], k);
            int64_t pb = L->parent[b];
            int64_t tmp[216];
            int nt = 0;
            for (int64_t e = Lp->nbr_start[pb]; e < Lp->nbr_start[pb + 1]; ++e) {
                int64_t q = Lp->nbr[e];
                for (int64_t c = Lp->child0[q]; c < Lp->child0[q + 1]; ++c) {
                    int64_t a[3];
                    demorton3(L->key[c], a);
                    int64_t m = 0;
                    for (int i = 0; i < 3; ++i) {
                        int64_t dd = a[i] > k[i] ? a[i] - k[i] : k[i] - a[i];
                        if (dd > m) m = dd;
                    }
                    if (m > 1) tmp[nt++] = c;
                }
            }
            qsort(tmp, (size_t)nt, sizeof(int64_t), cmp_i64);
            for (int i = 0; i < nt; ++i) ipush(&list, tmp[i]);
        }
        L->cous_start[L->nbox] = list.n;
        L->cous = list.v;
    }

    /* near-field ranges of every leaf box B of level l (reading R13): the points of all
     * neighbours of B at level l, and for each level d = 3 .. l-1 the points of the leaf
     * neighbours of B's ancestor at level d.  With leaves on level D only (the uniform
     * tree) these are the level-D neighbours of Algorithm 1's direct evaluations.  The
     * relation is symmetric, so the adjoint's direct sums use the same ranges. */
    for (int l = 3; l <= D; ++l) {
        olevel *L = &p->lev[l];
        L->near_start = malloc((size_t)(L->nbox + 1) * sizeof(int64_t));
        ivec lo = {0}, hi = {0};
        for (int64_t b = 0; b < L->nbox; ++b) {
            L->near_start[b] = lo.n;
            if (!L->leaf[b]) continue;
            ivec rg = {0};
            for (int64_t e = L->nbr_start[b]; e < L->nbr_start[b + 1]; ++e) {
                ipush(&rg, L->start[L->nbr[e]]);
                ipush(&rg, L->end[L->nbr[e]]);
            }
            int64_t a = b;
            for (int d = l - 1; d >= 3; --d) {
                a = p->lev[d + 1].parent[a];
                olevel *La = &p->lev[d];
                for (int64_t e = La->nbr_start[a]; e < La->nbr_start[a + 1]; ++e) {
                    int64_t q = La->nbr[e];
                    if (!La->leaf[q]) continue;
                    ipush(&rg, La->start[q]);
                    ipush(&rg, La->end[q]);
                }
            }
            qsort(rg.v, (size_t)(rg.n / 2), 2 * sizeof(int64_t), cmp_range);
            for (int64_t i = 0; i < rg.n; i += 2) {
                ipush(&lo, rg.v[i]);
                ipush(&hi, rg.v[i + 1]);
            }
            free(rg.v);
        }
        L->near_start[L->nbox] = lo.n;
        L->near_lo = lo.v ? lo.v : malloc(sizeof(int64_t));
        L->near_hi = hi.v ? hi.v : malloc(sizeof(int64_t));
    }

    /* cone levels (reading R5) and per-level tables */
    const double eta = sqrt(3.0) / 3.0;
    p->lev[D].ns = leaf_ns;
    p->lev[D].nc = leaf_nc;
    for (int d = D; d >= 4; --d) {
        int a = (2.0 * kappa * p->lev[d].H > 1.0) ? 2 : 1;
        p->lev[d - 1].ns = a * p->lev[d].ns;
        p->lev[d - 1].nc = a * p->lev[d].nc;
    }
    for (int d = 3; d <= D; ++d) {
        olevel *L = &p->lev[d];
        int ns = L->ns, nc = L->nc;
        L->h = sqrt(3.0) * 0.5 * L->H;
        L->ds = eta / (double)ns;
        L->dth = M_PI / (double)nc;
        L->cosk = malloc((size_t)(nc + 1) * sizeof(double));
        for (int k = 0; k <= nc; ++k) L->cosk[k] = cos(((double)k * M_PI) / (double)nc);
        L->nodeR = malloc((size_t)ns * Ps * sizeof(double));
        for (int g = 0; g < ns; ++g)
            for (int a = 0; a < Ps; ++a) {
                double s = L->ds * ((double)g + (1.0 + p->ts[a]) * 0.5);
                L->nodeR[g * Ps + a] = L->h / s;
            }
        size_t ntab = (size_t)(unsigned)nc * (size_t)(unsigned)Pang;
        L->sth = malloc(ntab * sizeof(double));
        L->cth = malloc(ntab * sizeof(double));
        for (int g = 0; g < nc; ++g)
            for (int b = 0; b < Pang; ++b) {
                double th = L->dth * ((double)g + (1.0 + p->ta[b]) * 0.5);
                L->sth[g * Pang + b] = sin(th);
                L->cth[g * Pang + b] = cos(th);
            }
        L->sph = malloc((size_t)2 * nc * Pang * sizeof(double));
        L->cph = malloc((size_t)2 * nc * Pang * sizeof(double));
        for (int g = 0; g < 2 * nc; ++g)
            for (int c = 0; c < Pang; ++c) {
                double ph = L->dth * ((double)g + (1.0 + p->ta[c]) * 0.5);
                L->sph[g * Pang + c] = sin(ph);
                L->cph[g * Pang + c] = cos(ph);
            }
    }

    /* relevant cone segments, top-down d = 3..D (Sec. 3.3.2, reading R7).  Boxes
     * of one level are independent once the parent level is done. */
    for (int d = 3; d <= D; ++d) {
        olevel *L = &p->lev[d];
        int64_t **box_ids = calloc((size_t)L->nbox, sizeof(int64_t *));
        int64_t *box_cnt = calloc((size_t)L->nbox, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t k = 0; k < L->nbox; ++k) {
            ivec ids = {0};
            double xk[3];
            box_center(p, d, L->key[k], xk);
            /* (i) cones containing a surface point of a cousin box */
            for (int64_t e = L->cous_start[k]; e < L->cous_start[k + 1]; ++e) {
                int64_t cb = L->cous[e];
                for (int64_t j = L->start[cb]; j < L->end[cb]; ++j)
                    ipush(&ids, cone_of(p, d, p->xs + 3 * j, xk, NULL, NULL));
            }
            /* (ii) cones containing an interpolation point of a relevant parent cone */
            if (d >= 4) {
                olevel *Lp = &p->lev[d - 1];
                int64_t pb = L->parent[k];
                int oct = (int)(L->key[k] & 7u);
                for (int64_t sl = Lp->act_start[pb]; sl < Lp->act_start[pb + 1]; ++sl)
                    for (int node = 0; node < p->P; ++node) {
                        double v[3];
                        node_rel_child(p, d, Lp->act_cone[sl], node, oct, v, NULL);
                        ipush(&ids, cone_of_vec(p, d, v, NULL, NULL));
                    }
            }
            box_cnt[k] = sort_unique(ids.v, ids.n);
            box_ids[k] = ids.v;
        }
        L->act_start = malloc((size_t)(L->nbox + 1) * sizeof(int64_t));
        int64_t tot = 0;
        for (int64_t k = 0; k < L->nbox; ++k) { L->act_start[k] = tot; tot += box_cnt[k]; }
        L->act_start[L->nbox] = tot;
        L->act_cone = malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int64_t));
        for (int64_t k = 0; k < L->nbox; ++k) {
            if (box_cnt[k]) memcpy(L->act_cone + L->act_start[k], box_ids[k], (size_t)box_cnt[k] * sizeof(int64_t));
            free(box_ids[k]);
        }
        free(box_ids);
        free(box_cnt);
        L->nact = tot;
    }
    return p;
}

void *oracle_plan_create(int64_t n, const double *pts, double kappa, int D, int Ps, int Pang,
                         int leaf_ns, int leaf_nc)
{
    return plan_create(n, pts, kappa, D, Ps, Pang, leaf_ns, leaf_nc, 0);
}

void *oracle_plan_create_adaptive(int64_t n, const double *pts, double kappa, int D, int Ps, int Pang,
                                  int leaf_ns, int leaf_nc, int64_t leaf_max)
{
    return plan_create(n, pts, kappa, D, Ps, Pang, leaf_ns, leaf_nc, leaf_max);
}

/* ------------------------------------------------------------------------- */
/* Evaluation (Algorithm 1).                                                  */
/* ------------------------------------------------------------------------- */

/* Interpolate the nrhs value sets of cone slot `sl` at local coordinates loc. */
static void interp(const oplan *p, const cplx *vals, const double *loc, int nrhs, cplx *out)
{
    double ws[64], wt[64], wp[64];
    lagrange(p->Ps, p->ts, loc[0], ws);
    lagrange(p->Pang, p->ta, loc[1], wt);
    lagrange(p->Pang, p->ta, loc[2], wp);
    for (int r = 0; r < nrhs; ++r) out[r] = 0;
    for (int a = 0; a < p->Ps; ++a)
        for (int b = 0; b < p->Pang; ++b)
            for (int c = 0; c < p->Pang; ++c) {
                double w = ws[a] * wt[b] * wp[c];
                int node = (a * p->Pang + b) * p->Pang + c;
                for (int r = 0; r < nrhs; ++r) out[r] += w * vals[(int64_t)node * nrhs + r];
            }
}

/* mode bit 1: near field (direct level-D sums); bit 2: far field (interpolation). */
int oracle_apply(void *h, int nrhs, const double *sigma_in, double *u_out, int mode)
{
    oplan *p = h;
    const int64_t n = p->n;
    const int D = p->D, P = p->P;
    const double kappa = p->kappa;
    const cplx *sigma = (const cplx *)sigma_in;
    cplx *u = (cplx *)u_out;
    /* densities in sorted order: a[j][r] */
    cplx *a = malloc((size_t)n * nrhs * sizeof(cplx));
    cplx *us = calloc((size_t)n * nrhs, sizeof(cplx));
    for (int64_t j = 0; j < n; ++j)
        for (int r = 0; r < nrhs; ++r) a[j * nrhs + r] = sigma[(int64_t)r * n + p->perm[j]];
    for (int d = 3; d <= D; ++d) {
        free(p->lev[d].F);
        p->lev[d].F = calloc((size_t)p->lev[d].nact * P * nrhs, sizeof(cplx));
        p->lev[d].cousin_evals = p->lev[d].upward_evals = 0;
    }
    p->nrhs_F = nrhs;
    int err = 0;
    int64_t near_pairs = 0;

    /* Direct evaluations: I_k at the surface points of the near field of every leaf
     * box (its level-D neighbours in the uniform tree, Algorithm 1; the ranges of
     * reading R13 in the adaptive tree); the pairs with target == source are skipped,
     * Eq. (field1). */
    if (mode & 1) {
        for (int l = 3; l <= D; ++l) {
            olevel *L = &p->lev[l];
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : near_pairs)
            for (int64_t b = 0; b < L->nbox; ++b) {
                if (!L->leaf[b]) continue;
                for (int64_t i = L->start[b]; i < L->end[b]; ++i) {
                    cplx acc[nrhs];
                    for (int r = 0; r < nrhs; ++r) acc[r] = 0;
                    for (int64_t e = L->near_start[b]; e < L->near_start[b + 1]; ++e)
                        for (int64_t j = L->near_lo[e]; j < L->near_hi[e]; ++j) {
                            if (j == i) continue;
                            cplx g = green(p->xs + 3 * i, p->xs + 3 * j, kappa);
                            for (int r = 0; r < nrhs; ++r) acc[r] += a[j * nrhs + r] * g;
                            near_pairs++;
                        }
                    for (int r = 0; r < nrhs; ++r) us[i * nrhs + r] += acc[r];
                }
            }
        }
    }
    p->near_pairs = near_pairs;

    if (mode & 2) {
        /* F_k at the interpolation points of every relevant cone of every leaf box k,
         * Eq. (I_k): level D in the uniform tree, any level >= 3 in the adaptive one. */
        for (int l = 3; l <= D; ++l) {
            olevel *L = &p->lev[l];
#pragma omp parallel for schedule(dynamic, 4)
            for (int64_t k = 0; k < L->nbox; ++k) {
                if (!L->leaf[k]) continue;
                double xk[3];
                box_center(p, l, L->key[k], xk);
                for (int64_t sl = L->act_start[k]; sl < L->act_start[k + 1]; ++sl)
                    for (int node = 0; node < P; ++node) {
                        double q[3];
                        node_pos(p, l, L->act_cone[sl], node, xk, q);
                        cplx *F = L->F + (sl * P + node) * nrhs;
                        for (int64_t j = L->start[k]; j < L->end[k]; ++j) {
                            cplx g = analytic_factor(q, xk, p->xs + 3 * j, kappa);
                            for (int r = 0; r < nrhs; ++r) F[r] += a[j * nrhs + r] * g;
                        }
                    }
            }
        }
        for (int d = D; d >= 3; --d) {
            olevel *Ld = &p->lev[d];
            int64_t cev = 0;
            /* cousin surface points: I_k^d(x) = G(x, x_k^d) * interpolated F_k^d(x).
             * Written per target x over the boxes k that have x as a cousin point;
             * the cousin relation is symmetric (b in M k  <=>  k in M b: both say the
             * parents are neighbours and the boxes are not), so this visits exactly
             * the (k, x) pairs of Algorithm 1, each target's terms in ascending k. */
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : cev, err)
            for (int64_t b = 0; b < Ld->nbox; ++b) {
                for (int64_t i = Ld->start[b]; i < Ld->end[b]; ++i) {
                    for (int64_t e = Ld->cous_start[b]; e < Ld->cous_start[b + 1]; ++e) {
                        int64_t k = Ld->cous[e];
                        double xk[3], loc[3];
                        box_center(p, d, Ld->key[k], xk);
                        int64_t cone = cone_of(p, d, p->xs + 3 * i, xk, NULL, loc);
                        int64_t sl = find_slot(Ld, k, cone);
                        if (sl < 0) { err++; continue; }
                        cplx v[nrhs];
                        interp(p, Ld->F + sl * P * nrhs, loc, nrhs, v);
                        cplx g = green(p->xs + 3 * i, xk, kappa);
                        for (int r = 0; r < nrhs; ++r) us[i * nrhs + r] += g * v[r];
                        cev++;
                    }
                }
            }
            Ld->cousin_evals = cev;
            if (d > 3) {
                /* parent interpolation points: F_j^{d-1}(x) += F_k^d(x) G(x,x_k^d)/G(x,x_j^{d-1})
                 * accumulated over the children k of j. */
                olevel *Lp = &p->lev[d - 1];
                int64_t uev = 0;
#pragma omp parallel for schedule(dynamic, 2) reduction(+ : uev, err)
                for (int64_t j = 0; j < Lp->nbox; ++j) {
                    for (int64_t sl = Lp->act_start[j]; sl < Lp->act_start[j + 1]; ++sl)
                        for (int node = 0; node < P; ++node) {
                            cplx *Fp = Lp->F + (sl * P + node) * nrhs;
                            for (int64_t k = Lp->child0[j]; k < Lp->child0[j + 1]; ++k) {
                                /* the point x relative to x_k^d, its cone and local coordinates */
                                double vk[3], loc[3];
                                double rj = node_rel_child(p, d, Lp->act_cone[sl], node, (int)(Ld->key[k] & 7u), vk, NULL);
                                int64_t cone = cone_of_vec(p, d, vk, NULL, loc);
                                int64_t csl = find_slot(Ld, k, cone);
                                if (csl < 0) { err++; continue; }
                                cplx v[nrhs];
                                interp(p, Ld->F + csl * P * nrhs, loc, nrhs, v);
                                /* G(x, x_k^d) / G(x, x_j^{d-1}) with |x - x_j| = rj, |x - x_k| = rk */
                                double rk = sqrt(vk[0] * vk[0] + vk[1] * vk[1] + vk[2] * vk[2]);
                                cplx fac = (rj / rk) * cexp(I * kappa * (rk - rj));
                                for (int r = 0; r < nrhs; ++r) Fp[r] += fac * v[r];
                                uev++;
                            }
                        }
                }
                Ld->upward_evals = uev;
            }
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int r = 0; r < nrhs; ++r) u[(int64_t)r * n + p->perm[j]] = us[j * nrhs + r];
    free(a);
    free(us);
    p->err = err;
    return err ? 1 : 0;
}

/*
 * Conjugate transpose of oracle_apply (mode bits as there).  With u = N a +
 * sum_d T_d F^d, F^D = L a, F^{d-1} = U_d F^d, the adjoint is
 *   Fbar^3 = T_3^H v,  Fbar^d = T_d^H v + U_d^H Fbar^{d-1} (d = 4..D),
 *   w = N^H v + L^H Fbar^D.
 * Every step below is the corresponding forward loop with the roles of source
 * and destination exchanged and every coefficient conjugated.
 */
int oracle_apply_adjoint(void *h, int nrhs, const double *v_in, double *w_out, int mode)
{
    oplan *p = h;
    const int64_t n = p->n;
    const int D = p->D, P = p->P;
    const double kappa = p->kappa;
    const cplx *vin = (const cplx *)v_in;
    cplx *w = (cplx *)w_out;
    cplx *v = malloc((size_t)n * nrhs * sizeof(cplx));
    cplx *ws = calloc((size_t)n * nrhs, sizeof(cplx));
    for (int64_t j = 0; j < n; ++j)
        for (int r = 0; r < nrhs; ++r) v[j * nrhs + r] = vin[(int64_t)r * n + p->perm[j]];
    for (int d = 3; d <= D; ++d) {
        free(p->lev[d].Fadj);
        p->lev[d].Fadj = calloc((size_t)p->lev[d].nact * P * nrhs, sizeof(cplx));
    }
    int err = 0;
    if (mode & 1) {
        /* N^H: source j gathers conj(G(x_i, x_j)) v_i over the targets i of its own
         * near-field ranges (the near relation is symmetric). */
        for (int l = 3; l <= D; ++l) {
            olevel *L = &p->lev[l];
#pragma omp parallel for schedule(dynamic, 8)
            for (int64_t b = 0; b < L->nbox; ++b) {
                if (!L->leaf[b]) continue;
                for (int64_t j = L->start[b]; j < L->end[b]; ++j) {
                    cplx acc[nrhs];
                    for (int r = 0; r < nrhs; ++r) acc[r] = 0;
                    for (int64_t e = L->near_start[b]; e < L->near_start[b + 1]; ++e)
                        for (int64_t i = L->near_lo[e]; i < L->near_hi[e]; ++i) {
                            if (i == j) continue;
                            cplx g = conj(green(p->xs + 3 * i, p->xs + 3 * j, kappa));
                            for (int r = 0; r < nrhs; ++r) acc[r] += v[i * nrhs + r] * g;
                        }
                    for (int r = 0; r < nrhs; ++r) ws[j * nrhs + r] += acc[r];
                }
            }
        }
    }
    if (mode & 2) {
        for (int d = 3; d <= D; ++d) {
            olevel *Ld = &p->lev[d];
            /* T_d^H: each source box k collects from its cousin points x:
             * Fbar_k[slot][node] += conj(G(x, x_k) L_node(x)) v(x). */
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : err)
            for (int64_t k = 0; k < Ld->nbox; ++k) {
                double xk[3];
                box_center(p, d, Ld->key[k], xk);
                for (int64_t e = Ld->cous_start[k]; e < Ld->cous_start[k + 1]; ++e) {
                    int64_t b = Ld->cous[e];
                    for (int64_t i = Ld->start[b]; i < Ld->end[b]; ++i) {
                        double loc[3], wsd[64], wt[64], wp[64];
                        int64_t cone = cone_of(p, d, p->xs + 3 * i, xk, NULL, loc);
                        int64_t sl = find_slot(Ld, k, cone);
                        if (sl < 0) { err++; continue; }
                        lagrange(p->Ps, p->ts, loc[0], wsd);
                        lagrange(p->Pang, p->ta, loc[1], wt);
                        lagrange(p->Pang, p->ta, loc[2], wp);
                        cplx g = conj(green(p->xs + 3 * i, xk, kappa));
                        for (int a = 0; a < p->Ps; ++a)
                            for (int bb = 0; bb < p->Pang; ++bb)
                                for (int c = 0; c < p->Pang; ++c) {
                                    int node = (a * p->Pang + bb) * p->Pang + c;
                                    double wgt = wsd[a] * wt[bb] * wp[c];
                                    for (int r = 0; r < nrhs; ++r)
                                        Ld->Fadj[(sl * P + node) * nrhs + r] += wgt * g * v[i * nrhs + r];
                                }
                    }
                }
            }
            /* U_d^H (d >= 4): each child box k receives from the interpolation
             * points of its parent's relevant cones. */
            if (d >= 4) {
                olevel *Lp = &p->lev[d - 1];
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : err)
                for (int64_t k = 0; k < Ld->nbox; ++k) {
                    int64_t j = Ld->parent[k];
                    int oct = (int)(Ld->key[k] & 7u);
                    for (int64_t sl = Lp->act_start[j]; sl < Lp->act_start[j + 1]; ++sl)
                        for (int node = 0; node < P; ++node) {
                            double vk[3], loc[3], wsd[64], wt[64], wp[64];
                            double rj = node_rel_child(p, d, Lp->act_cone[sl], node, oct, vk, NULL);
                            int64_t cone = cone_of_vec(p, d, vk, NULL, loc);
                            int64_t csl = find_slot(Ld, k, cone);
                            if (csl < 0) { err++; continue; }
                            lagrange(p->Ps, p->ts, loc[0], wsd);
                            lagrange(p->Pang, p->ta, loc[1], wt);
                            lagrange(p->Pang, p->ta, loc[2], wp);
                            double rk = sqrt(vk[0] * vk[0] + vk[1] * vk[1] + vk[2] * vk[2]);
                            cplx fac = conj((rj / rk) * cexp(I * kappa * (rk - rj)));
                            const cplx *src = Lp->Fadj + (sl * P + node) * nrhs;
                            for (int a = 0; a < p->Ps; ++a)
                                for (int bb = 0; bb < p->Pang; ++bb)
                                    for (int c = 0; c < p->Pang; ++c) {
                                        int cn = (a * p->Pang + bb) * p->Pang + c;
                                        double wgt = wsd[a] * wt[bb] * wp[c];
                                        for (int r = 0; r < nrhs; ++r)
                                            Ld->Fadj[(csl * P + cn) * nrhs + r] += wgt * fac * src[r];
                                    }
                        }
                }
            }
        }
        /* L^H: each source gathers conj(g(q, x')) Fbar over its leaf's cone nodes */
        for (int l = 3; l <= D; ++l) {
            olevel *L = &p->lev[l];
#pragma omp parallel for schedule(dynamic, 4)
            for (int64_t k = 0; k < L->nbox; ++k) {
                if (!L->leaf[k]) continue;
                double xk[3];
                box_center(p, l, L->key[k], xk);
                for (int64_t j = L->start[k]; j < L->end[k]; ++j) {
                    cplx acc[nrhs];
                    for (int r = 0; r < nrhs; ++r) acc[r] = 0;
                    for (int64_t sl = L->act_start[k]; sl < L->act_start[k + 1]; ++sl)
                        for (int node = 0; node < P; ++node) {
                            double q[3];
                            node_pos(p, l, L->act_cone[sl], node, xk, q);
                            cplx g = conj(analytic_factor(q, xk, p->xs + 3 * j, kappa));
                            for (int r = 0; r < nrhs; ++r) acc[r] += g * L->Fadj[(sl * P + node) * nrhs + r];
                        }
                    for (int r = 0; r < nrhs; ++r) ws[j * nrhs + r] += acc[r];
                }
            }
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int r = 0; r < nrhs; ++r) w[(int64_t)r * n + p->perm[j]] = ws[j * nrhs + r];
    free(v);
    free(ws);
    return err ? 1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Introspection for tests.                                                   */
/* ------------------------------------------------------------------------- */

/* info: [n, D, P, Ps, Pang, near_pairs] */
void oracle_plan_info(void *h, int64_t *info)
{
    oplan *p = h;
    info[0] = p->n; info[1] = p->D; info[2] = p->P; info[3] = p->Ps; info[4] = p->Pang;
    info[5] = p->near_pairs;
}

/* geometry: [H1, corner0, corner1, corner2] */
void oracle_plan_geometry(void *h, double *g)
{
    oplan *p = h;
    g[0] = p->H1; g[1] = p->corner[0]; g[2] = p->corner[1]; g[3] = p->corner[2];
}

/* level info: [nbox, nnbr, ncous, nact, ns, nc, cousin_evals, upward_evals] */
void oracle_level_info(void *h, int d, int64_t *info)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    info[0] = L->nbox;
    info[1] = L->nbr_start ? L->nbr_start[L->nbox] : 0;
    info[2] = L->cous_start ? L->cous_start[L->nbox] : 0;
    info[3] = L->nact;
    info[4] = L->ns;
    info[5] = L->nc;
    info[6] = L->cousin_evals;
    info[7] = L->upward_evals;
}

/* level scalars: [H, h, ds, dth] */
void oracle_level_params(void *h, int d, double *v)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    v[0] = L->H; v[1] = L->h; v[2] = L->ds; v[3] = L->dth;
}

void oracle_get_perm(void *h, int64_t *perm)
{
    oplan *p = h;
    memcpy(perm, p->perm, (size_t)p->n * sizeof(int64_t));
}

void oracle_get_boxes(void *h, int d, uint64_t *keys, int64_t *start)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    memcpy(keys, L->key, (size_t)L->nbox * sizeof(uint64_t));
    memcpy(start, L->start, (size_t)(L->nbox + 1) * sizeof(int64_t));
}

/* end[nbox] and leaf[nbox] of level d (adaptive trees: the point ranges of the boxes
 * are [start[b], end[b]) and leaf boxes are not subdivided) */
void oracle_get_box_ends(void *h, int d, int64_t *end, int64_t *leaf)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    for (int64_t b = 0; b < L->nbox; ++b) { end[b] = L->end[b]; leaf[b] = L->leaf[b]; }
}

/* near-field ranges of the leaf boxes of level d >= 3: start[nbox+1] into lo/hi */
int64_t oracle_get_near(void *h, int d, int64_t *start, int64_t *lo, int64_t *hi)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    int64_t m = L->near_start[L->nbox];
    if (start) {
        for (int64_t b = 0; b <= L->nbox; ++b) start[b] = L->near_start[b];
        for (int64_t e = 0; e < m; ++e) { lo[e] = L->near_lo[e]; hi[e] = L->near_hi[e]; }
    }
    return m;
}

/* leaf level of every point, in sorted (Morton) order */
void oracle_get_point_levels(void *h, int64_t *lev)
{
    oplan *p = h;
    for (int64_t j = 0; j < p->n; ++j) lev[j] = p->ptlev[j];
}

void oracle_get_neighbors(void *h, int d, int64_t *start, int64_t *list)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    memcpy(start, L->nbr_start, (size_t)(L->nbox + 1) * sizeof(int64_t));
    memcpy(list, L->nbr, (size_t)L->nbr_start[L->nbox] * sizeof(int64_t));
}

void oracle_get_cousins(void *h, int d, int64_t *start, int64_t *list)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    memcpy(start, L->cous_start, (size_t)(L->nbox + 1) * sizeof(int64_t));
    memcpy(list, L->cous, (size_t)L->cous_start[L->nbox] * sizeof(int64_t));
}

void oracle_get_active(void *h, int d, int64_t *start, int64_t *cones)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    memcpy(start, L->act_start, (size_t)(L->nbox + 1) * sizeof(int64_t));
    memcpy(cones, L->act_cone, (size_t)L->nact * sizeof(int64_t));
}

/* F values of level d after the last apply: [nact][P][nrhs] complex */
void oracle_get_F(void *h, int d, double *out)
{
    oplan *p = h;
    olevel *L = &p->lev[d];
    memcpy(out, L->F, (size_t)L->nact * p->P * p->nrhs_F * sizeof(cplx));
}

/* cone of point y w.r.t. centre c at level d: g[0..2] cell indices, g[3] linear id;
 * loc: local coordinates */
void oracle_cone_of(void *h, int d, const double *y, const double *c, int64_t *g, double *loc)
{
    oplan *p = h;
    g[3] = cone_of(p, d, y, c, g, loc);
}

/* position of node `node` of cone `cone` around centre x at level d */
double oracle_node_pos(void *h, int d, int64_t cone, int node, const double *x, double *q)
{
    return node_pos(h, d, cone, node, x, q);
}

void oracle_box_center(void *h, int d, uint64_t key, double *c) { box_center(h, d, key, c); }

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
