/*
 * FP64 CPU oracle for the explicit DVM Boltzmann step on a quad/octree.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares
 * no code with the CUDA library.
 *
 * Paper: Zabelok, Arslanbekov, Kolobov, "Adaptive Kinetic-Fluid Solvers for
 * Heterogeneous Computing Architectures".
 *   - tree mesh, 2:1 balance for direct and diagonal neighbours ... Sec. 2.1
 *   - Morton (N-order) ordering of the leaves ...................... Sec. 2.1
 *   - discrete velocities at cell centres of a uniform grid ........ Sec. 3
 *   - finite-volume advection ........................... Sec. 3.1, Eq. 2
 *   - 8 sign groups of velocity points, stored contiguously ........ Sec. 3.1
 *   - discrete collision integral, B, C, conservative correction Eqs. 3-6
 *   - BGK relaxation form ........................................... Sec. 4
 * Where the paper leaves a choice open, the reading used here is the one
 * listed with the library's design notes (first-order upwind fluxes,
 * CFL definition, Lie splitting, seeded hard-sphere trials, the DVM-BGK
 * collision frequency, boundary kinds).
 */
#include "dvm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int lev;
    int32_t i[3];      /* integer box coordinates at the box's own level */
    uint64_t key;      /* Morton key of the anchor at the deepest level  */
    uint8_t solid;
} leaf_t;

struct orc_problem {
    orc_tree_spec spec;
    int L;
    int64_t nleaves;
    leaf_t *lv;
    int64_t ncells;
    int64_t *cell_of_leaf;
    int64_t *leaf_of_cell;
    /* interior faces */
    int64_t nf;
    int64_t *fm, *fp;
    uint8_t *fax;
    double *farea;
    /* boundary faces */
    int64_t nbf;
    int64_t *bl, *bother;
    uint8_t *bax, *bside, *bkind;
    double *barea;
    /* faces touching each cell, interior faces first, each list in face order:
     * entry >= 0 is interior face q, entry < 0 is boundary face -1-q */
    int64_t *cf_start, *cf_list;
    /* velocity grid */
    int n[3];
    double lo[3], hi[3], h[3], dV;
    int64_t nv;
    double *xi;
    int32_t *k;
    int64_t *mirror[3];
    /* state */
    double *f;
    double fs_rho, fs_u[3], fs_T;
    double *finf;
    /* hard-sphere tables (CSR over nodes) */
    int hs_trials;
    int64_t hs_nkept;
    int64_t *hs_start;
    int32_t *hs_gam, *hs_l, *hs_m;
    double *hs_b;
    int64_t hs_discarded;
    /* LBM velocity set (0: a DVM grid) and its weights */
    int lattice;
    double *lw;
};

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014): output n of the stream whose state
 * starts at `seed` and advances by the golden-ratio increment each draw.   */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* the number of OpenMP threads of later loops (timing only) */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

uint64_t orc_splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + (n + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double unif53(uint64_t seed, uint64_t n)
{
    return (double)(orc_splitmix64(seed, n) >> 11) * 0x1.0p-53;
}

/* ------------------------------------------------------------------------ */
/* Velocity grid.  Nodes are cell centres of a uniform grid (Sec. 3):
 * xi_d(k) = lo_d + (k + 1/2) h_d with h_d = (hi_d - lo_d)/n_d.  The nodes are
 * grouped by the signs of their three components (Sec. 3.1 step 1): group
 * o = 4[xi_x>0] + 2[xi_y>0] + [xi_z>0], so group 0 is (-,-,-) and group 1 is
 * (-,-,+).  Inside a group the nodes are ordered lexicographically by the
 * distance index m_d (m_d = 0 nearest to zero), z fastest. */
int64_t orc_vgrid_size(const int n[3])
{
    return (int64_t)n[0] * n[1] * n[2];
}

static int axis_index(int n, int positive, int m)
{
    return positive ? n / 2 + m : n / 2 - 1 - m;
}

int orc_vgrid(const int n[3], const double lo[3], const double hi[3],
              double *xi, int32_t *k, double *dV)
{
    for (int d = 0; d < 3; d++)
        if (n[d] <= 0 || n[d] % 2 != 0 || !(hi[d] > lo[d])) return -1;
    double h[3];
    for (int d = 0; d < 3; d++) h[d] = (hi[d] - lo[d]) / n[d];
    int half[3] = {n[0] / 2, n[1] / 2, n[2] / 2};
    int64_t v = 0;
    for (int o = 0; o < 8; o++) {
        int pos[3] = {(o >> 2) & 1, (o >> 1) & 1, o & 1};
        for (int mx = 0; mx < half[0]; mx++)
            for (int my = 0; my < half[1]; my++)
                for (int mz = 0; mz < half[2]; mz++) {
                    int kk[3] = {axis_index(n[0], pos[0], mx),
                                 axis_index(n[1], pos[1], my),
                                 axis_index(n[2], pos[2], mz)};
                    for (int d = 0; d < 3; d++) {
                        if (xi) xi[3 * v + d] = lo[d] + ((double)kk[d] + 0.5) * h[d];
                        if (k) k[3 * v + d] = kk[d];
                    }
                    v++;
                }
    }
    if (dV) *dV = h[0] * h[1] * h[2];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tree (Sec. 2.1): boxes obtained by repeated halving; leaves are cells.    */

static uint64_t morton(int dim, int L, const int32_t a[3])
{
    uint64_t key = 0;
    for (int b = 0; b < L; b++)
        for (int d = 0; d < dim; d++)
            key |= (uint64_t)((a[d] >> b) & 1) << (dim * b + d);
    return key;
}

static void set_key(leaf_t *x, int dim, int L)
{
    int32_t a[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) a[d] = x->i[d] << (L - x->lev);
    x->key = morton(dim, L, a);
}

static int periodic_axis(const orc_tree_spec *s, int d)
{
    return s->bc[2 * d] == ORC_BC_PERIODIC;
}

/* squared distance from point c to the box, and to its farthest point */
static double box_dmin2(const orc_tree_spec *s, int lev, const int32_t i[3])
{
    double h = ldexp(1.0, -lev), d2 = 0.0;
    for (int d = 0; d < s->dim; d++) {
        double lo = i[d] * h, hi = (i[d] + 1) * h, t = 0.0;
        if (s->c[d] < lo) t = lo - s->c[d];
        else if (s->c[d] > hi) t = s->c[d] - hi;
        d2 += t * t;
    }
    return d2;
}

static double box_dmax2(const orc_tree_spec *s, int lev, const int32_t i[3])
{
    double h = ldexp(1.0, -lev), d2 = 0.0;
    for (int d = 0; d < s->dim; d++) {
        double a = fabs(i[d] * h - s->c[d]), b = fabs((i[d] + 1) * h - s->c[d]);
        double t = a > b ? a : b;
        d2 += t * t;
    }
    return d2;
}

static int refine_pred(const orc_tree_spec *s, const leaf_t *x)
{
    if (x->lev >= s->max_level) return 0;
    if (s->pred == ORC_PRED_BALL) {
        return box_dmin2(s, x->lev, x->i) <= s->r * s->r;
    }
    if (s->pred == ORC_PRED_SHELL) {
        double h = ldexp(1.0, -x->lev);
        double rp = s->r + s->beta * h, rm = s->r - s->beta * h;
        if (!(box_dmin2(s, x->lev, x->i) <= rp * rp)) return 0;
        return rm <= 0.0 || box_dmax2(s, x->lev, x->i) >= rm * rm;
    }
    return 0;
}

static int is_solid(const orc_tree_spec *s, const leaf_t *x)
{
    if (!s->solid) return 0;
    double h = ldexp(1.0, -x->lev), d2 = 0.0;
    for (int d = 0; d < s->dim; d++) {
        double t = (x->i[d] + 0.5) * h - s->c[d];
        d2 += t * t;
    }
    return d2 < s->r * s->r;
}

static int cmp_leaf(const void *a, const void *b)
{
    uint64_t x = ((const leaf_t *)a)->key, y = ((const leaf_t *)b)->key;
    return x < y ? -1 : x > y;
}

/* index of the leaf containing the deepest-level cell with Morton key `key`:
 * the last leaf whose anchor key is <= key (leaves cover contiguous key
 * ranges in Morton order). */
static int64_t locate(const leaf_t *lv, int64_t n, uint64_t key)
{
    int64_t lo = 0, hi = n - 1, ans = -1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (lv[mid].key <= key) { ans = mid; lo = mid + 1; }
        else hi = mid - 1;
    }
    return ans;
}

static int64_t locate_cell(const leaf_t *lv, int64_t n, int dim, int L,
                           int lev, const int32_t c[3])
{
    int32_t a[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) a[d] = c[d] << (L - lev);
    return locate(lv, n, morton(dim, L, a));
}

typedef struct { leaf_t *v; int64_t n, cap; } leafvec;

static int push(leafvec *lv, leaf_t x)
{
    if (lv->n == lv->cap) {
        int64_t nc = lv->cap ? 2 * lv->cap : 1024;
        leaf_t *nv = (leaf_t *)realloc(lv->v, (size_t)nc * sizeof(leaf_t));
        if (!nv) return -1;
        lv->v = nv;
        lv->cap = nc;
    }
    lv->v[lv->n++] = x;
    return 0;
}

static int push_children(leafvec *out, const leaf_t *x, int dim, int L)
{
    int nch = 1 << dim;
    for (int c = 0; c < nch; c++) {
        leaf_t y;
        memset(&y, 0, sizeof y);
        y.lev = x->lev + 1;
        for (int d = 0; d < dim; d++) y.i[d] = 2 * x->i[d] + ((c >> d) & 1);
        set_key(&y, dim, L);
        if (push(out, y)) return -1;
    }
    return 0;
}

/* 1 if some leaf touching x (across a face, edge or corner, periodic sides
 * wrapped) is more than one level finer than x. */
static int violates_balance(const orc_tree_spec *s, int L, const leaf_t *lv,
                            int64_t n, const leaf_t *x)
{
    int dim = s->dim, lev = x->lev + 2;
    if (lev > L) return 0;
    int32_t N = (int32_t)1 << lev;
    int lo3 = dim == 3 ? -1 : 0, hi3 = dim == 3 ? 4 : 0;
    for (int oz = lo3; oz <= hi3; oz++)
        for (int oy = -1; oy <= 4; oy++)
            for (int ox = -1; ox <= 4; ox++) {
                int off[3] = {ox, oy, oz};
                int inside = 1;
                for (int d = 0; d < dim; d++)
                    if (off[d] < 0 || off[d] > 3) inside = 0;
                if (inside) continue;
                int32_t c[3] = {0, 0, 0};
                int ok = 1;
                for (int d = 0; d < dim; d++) {
                    c[d] = 4 * x->i[d] + off[d];
                    if (c[d] < 0 || c[d] >= N) {
                        if (periodic_axis(s, d)) c[d] = (c[d] + N) % N;
                        else ok = 0;
                    }
                }
                if (!ok) continue;
                int64_t b = locate_cell(lv, n, dim, L, lev, c);
                if (b >= 0 && lv[b].lev >= lev) return 1;
            }
    return 0;
}

static int check_spec(const orc_tree_spec *s)
{
    if (s->dim != 2 && s->dim != 3) return -1;
    if (s->base_level < 1 || s->max_level < s->base_level) return -1;
    if (s->max_level * s->dim > 63) return -1;
    for (int d = 0; d < s->dim; d++)
        if ((s->bc[2 * d] == ORC_BC_PERIODIC) != (s->bc[2 * d + 1] == ORC_BC_PERIODIC))
            return -1;
    return 0;
}

/* 2:1 balance for direct and diagonal neighbours, to a fixpoint: every leaf
 * that touches a leaf two or more levels finer is split; the result is
 * sorted in Morton order. */
static int balance_fixpoint(const orc_tree_spec *s, leafvec *cur)
{
    int dim = s->dim, L = s->max_level;
    for (;;) {
        qsort(cur->v, (size_t)cur->n, sizeof(leaf_t), cmp_leaf);
        char *mark = (char *)calloc((size_t)cur->n + 1, 1);
        if (!mark) return -1;
        int64_t nmark = 0;
        for (int64_t a = 0; a < cur->n; a++)
            if (violates_balance(s, L, cur->v, cur->n, &cur->v[a])) { mark[a] = 1; nmark++; }
        if (nmark == 0) { free(mark); break; }
        leafvec nxt = {0, 0, 0};
        for (int64_t a = 0; a < cur->n; a++) {
            if (mark[a]) { if (push_children(&nxt, &cur->v[a], dim, L)) return -1; }
            else if (push(&nxt, cur->v[a])) return -1;
        }
        free(mark);
        free(cur->v);
        *cur = nxt;
    }
    return 0;
}

static int build_tree(const orc_tree_spec *s, leafvec *out)
{
    int dim = s->dim, L = s->max_level;
    leafvec cur = {0, 0, 0};
    int32_t N = (int32_t)1 << s->base_level;
    int32_t nz = dim == 3 ? N : 1;
    for (int32_t z = 0; z < nz; z++)
        for (int32_t y = 0; y < N; y++)
            for (int32_t x = 0; x < N; x++) {
                leaf_t t;
                memset(&t, 0, sizeof t);
                t.lev = s->base_level;
                t.i[0] = x; t.i[1] = y; t.i[2] = z;
                set_key(&t, dim, L);
                if (push(&cur, t)) return -1;
            }
    /* refinement by the predicate, to a fixpoint */
    for (;;) {
        leafvec nxt = {0, 0, 0};
        int changed = 0;
        for (int64_t a = 0; a < cur.n; a++) {
            if (refine_pred(s, &cur.v[a])) {
                if (push_children(&nxt, &cur.v[a], dim, L)) return -1;
                changed = 1;
            } else if (push(&nxt, cur.v[a])) return -1;
        }
        free(cur.v);
        cur = nxt;
        if (!changed) break;
    }
    if (balance_fixpoint(s, &cur)) return -1;
    for (int64_t a = 0; a < cur.n; a++) cur.v[a].solid = (uint8_t)is_solid(s, &cur.v[a]);
    *out = cur;
    return 0;
}

int orc_build_tree(const orc_tree_spec *spec, int64_t cap, int64_t *n,
                   uint64_t *keys, uint8_t *levels, uint8_t *solid)
{
    if (check_spec(spec)) return -1;
    leafvec t;
    if (build_tree(spec, &t)) return -2;
    *n = t.n;
    if (t.n > cap) { free(t.v); return cap == 0 ? 0 : -3; }
    for (int64_t a = 0; a < t.n; a++) {
        if (keys) keys[a] = t.v[a].key;
        if (levels) levels[a] = (uint8_t)t.v[a].lev;
        if (solid) solid[a] = t.v[a].solid;
    }
    free(t.v);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Faces.  One interior face per fine subface between two fluid leaves,
 * recorded from its minus side; boundary faces on the domain sides and
 * towards solid leaves.  Area = (edge of the finer box)^(dim-1).            */

typedef struct { int64_t m, p; uint8_t ax; double area; uint64_t km, kp; } iface_t;
typedef struct { int64_t l, o; uint8_t ax, side, kind; double area; uint64_t kl, ko; } bface_t;

static int cmp_iface(const void *a, const void *b)
{
    const iface_t *x = (const iface_t *)a, *y = (const iface_t *)b;
    if (x->ax != y->ax) return x->ax < y->ax ? -1 : 1;
    if (x->km != y->km) return x->km < y->km ? -1 : 1;
    if (x->kp != y->kp) return x->kp < y->kp ? -1 : 1;
    return 0;
}

static int cmp_bface(const void *a, const void *b)
{
    const bface_t *x = (const bface_t *)a, *y = (const bface_t *)b;
    if (x->kind != y->kind) return x->kind < y->kind ? -1 : 1;
    if (x->ax != y->ax) return x->ax < y->ax ? -1 : 1;
    if (x->side != y->side) return x->side < y->side ? -1 : 1;
    if (x->kl != y->kl) return x->kl < y->kl ? -1 : 1;
    if (x->ko != y->ko) return x->ko < y->ko ? -1 : 1;
    return 0;
}

static int build_faces(orc_problem *p)
{
    const orc_tree_spec *s = &p->spec;
    int dim = s->dim, L = p->L;
    int64_t icap = 1024, bcap = 1024, ni = 0, nb = 0;
    iface_t *fi = (iface_t *)malloc((size_t)icap * sizeof(iface_t));
    bface_t *fb = (bface_t *)malloc((size_t)bcap * sizeof(bface_t));
    if (!fi || !fb) return -1;
    for (int64_t a = 0; a < p->nleaves; a++) {
        const leaf_t *A = &p->lv[a];
        if (A->solid) continue;
        for (int d = 0; d < dim; d++)
            for (int side = 0; side < 2; side++) {
                int32_t N = (int32_t)1 << A->lev;
                int32_t c[3] = {A->i[0], A->i[1], A->i[2]};
                c[d] += side ? 1 : -1;
                if (c[d] < 0 || c[d] >= N) {
                    if (periodic_axis(s, d)) c[d] = (c[d] + N) % N;
                    else {
                        if (nb == bcap) { bcap *= 2; fb = (bface_t *)realloc(fb, (size_t)bcap * sizeof(bface_t)); }
                        bface_t t = {a, -1, (uint8_t)d, (uint8_t)side, (uint8_t)s->bc[2 * d + side],
                                     ldexp(1.0, -A->lev * (dim - 1)), A->key, 0};
                        fb[nb++] = t;
                        continue;
                    }
                }
                int64_t nbrs[4];
                int nn = 0;
                double area;
                int64_t b = locate_cell(p->lv, p->nleaves, dim, L, A->lev, c);
                if (p->lv[b].lev <= A->lev) {
                    nbrs[nn++] = b;
                    area = ldexp(1.0, -A->lev * (dim - 1));
                } else {
                    /* the finer neighbours: children of c on the side facing A */
                    int nsub = 1 << (dim - 1);
                    for (int t = 0; t < nsub; t++) {
                        int32_t cc[3] = {0, 0, 0};
                        int bit = 0;
                        for (int e = 0; e < dim; e++) {
                            if (e == d) cc[e] = 2 * c[e] + (side ? 0 : 1);
                            else cc[e] = 2 * c[e] + ((t >> bit++) & 1);
                        }
                        int64_t bb = locate_cell(p->lv, p->nleaves, dim, L, A->lev + 1, cc);
                        if (p->lv[bb].lev != A->lev + 1) { free(fi); free(fb); return -2; }
                        nbrs[nn++] = bb;
                    }
                    area = ldexp(1.0, -(A->lev + 1) * (dim - 1));
                }
                for (int t = 0; t < nn; t++) {
                    int64_t bb = nbrs[t];
                    if (p->lv[bb].solid) {
                        if (nb == bcap) { bcap *= 2; fb = (bface_t *)realloc(fb, (size_t)bcap * sizeof(bface_t)); }
                        bface_t w = {a, bb, (uint8_t)d, (uint8_t)side, ORC_BC_WALL, area,
                                     A->key, p->lv[bb].key};
                        fb[nb++] = w;
                    } else if (side == 1) {
                        if (ni == icap) { icap *= 2; fi = (iface_t *)realloc(fi, (size_t)icap * sizeof(iface_t)); }
                        iface_t w = {a, bb, (uint8_t)d, area, A->key, p->lv[bb].key};
                        fi[ni++] = w;
                    }
                }
            }
    }
    qsort(fi, (size_t)ni, sizeof(iface_t), cmp_iface);
    qsort(fb, (size_t)nb, sizeof(bface_t), cmp_bface);
    p->nf = ni;
    p->fm = (int64_t *)malloc((size_t)(ni + 1) * sizeof(int64_t));
    p->fp = (int64_t *)malloc((size_t)(ni + 1) * sizeof(int64_t));
    p->fax = (uint8_t *)malloc((size_t)(ni + 1));
    p->farea = (double *)malloc((size_t)(ni + 1) * sizeof(double));
    for (int64_t q = 0; q < ni; q++) {
        p->fm[q] = fi[q].m; p->fp[q] = fi[q].p; p->fax[q] = fi[q].ax; p->farea[q] = fi[q].area;
    }
    p->nbf = nb;
    p->bl = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
    p->bother = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
    p->bax = (uint8_t *)malloc((size_t)(nb + 1));
    p->bside = (uint8_t *)malloc((size_t)(nb + 1));
    p->bkind = (uint8_t *)malloc((size_t)(nb + 1));
    p->barea = (double *)malloc((size_t)(nb + 1) * sizeof(double));
    for (int64_t q = 0; q < nb; q++) {
        p->bl[q] = fb[q].l; p->bother[q] = fb[q].o; p->bax[q] = fb[q].ax;
        p->bside[q] = fb[q].side; p->bkind[q] = fb[q].kind; p->barea[q] = fb[q].area;
    }
    free(fi);
    free(fb);
    /* per-cell face lists */
    p->cf_start = (int64_t *)calloc((size_t)(p->ncells + 1), sizeof(int64_t));
    p->cf_list = (int64_t *)malloc((size_t)(2 * ni + nb + 1) * sizeof(int64_t));
    for (int64_t q = 0; q < ni; q++) {
        p->cf_start[p->cell_of_leaf[p->fm[q]] + 1]++;
        p->cf_start[p->cell_of_leaf[p->fp[q]] + 1]++;
    }
    for (int64_t q = 0; q < nb; q++) p->cf_start[p->cell_of_leaf[p->bl[q]] + 1]++;
    for (int64_t c = 0; c < p->ncells; c++) p->cf_start[c + 1] += p->cf_start[c];
    int64_t *fill = (int64_t *)malloc((size_t)(p->ncells + 1) * sizeof(int64_t));
    memcpy(fill, p->cf_start, (size_t)(p->ncells + 1) * sizeof(int64_t));
    for (int64_t q = 0; q < ni; q++) {
        int64_t a = p->cell_of_leaf[p->fm[q]], b = p->cell_of_leaf[p->fp[q]];
        p->cf_list[fill[a]++] = q;
        p->cf_list[fill[b]++] = q;
    }
    for (int64_t q = 0; q < nb; q++) {
        int64_t a = p->cell_of_leaf[p->bl[q]];
        p->cf_list[fill[a]++] = -1 - q;
    }
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------------ */

static double maxwellian(double rho, const double u[3], double T, const double xi[3])
{
    double q = 0.0;
    for (int d = 0; d < 3; d++) q += (xi[d] - u[d]) * (xi[d] - u[d]);
    return rho * pow(2.0 * M_PI * T, -1.5) * exp(-q / (2.0 * T));
}

/* the tree, its cells and faces; no velocity set yet */
static orc_problem *create_tree(const orc_tree_spec *spec)
{
    if (check_spec(spec)) return NULL;
    orc_problem *p = (orc_problem *)calloc(1, sizeof(orc_problem));
    if (!p) return NULL;
    p->spec = *spec;
    p->L = spec->max_level;
    leafvec t;
    if (build_tree(spec, &t)) { free(p); return NULL; }
    p->lv = t.v;
    p->nleaves = t.n;
    p->cell_of_leaf = (int64_t *)malloc((size_t)t.n * sizeof(int64_t));
    p->leaf_of_cell = (int64_t *)malloc((size_t)t.n * sizeof(int64_t));
    for (int64_t a = 0; a < t.n; a++) {
        if (p->lv[a].solid) p->cell_of_leaf[a] = -1;
        else { p->cell_of_leaf[a] = p->ncells; p->leaf_of_cell[p->ncells++] = a; }
    }
    if (build_faces(p)) { orc_destroy(p); return NULL; }
    return p;
}

static orc_problem *create_grid(const orc_tree_spec *spec, const int n[3], const double lo[3],
                                const double hi[3], int with_f)
{
    orc_problem *p = create_tree(spec);
    if (!p) return NULL;
    for (int d = 0; d < 3; d++) { p->n[d] = n[d]; p->lo[d] = lo[d]; p->hi[d] = hi[d]; }
    p->nv = orc_vgrid_size(n);
    p->xi = (double *)malloc((size_t)p->nv * 3 * sizeof(double));
    p->k = (int32_t *)malloc((size_t)p->nv * 3 * sizeof(int32_t));
    if (orc_vgrid(n, lo, hi, p->xi, p->k, &p->dV)) { orc_destroy(p); return NULL; }
    for (int d = 0; d < 3; d++) p->h[d] = (hi[d] - lo[d]) / n[d];
    /* mirror maps: the node whose component d is reflected (k -> n-1-k) */
    int64_t *idx = (int64_t *)malloc((size_t)p->nv * sizeof(int64_t));
    for (int64_t v = 0; v < p->nv; v++) {
        const int32_t *kk = &p->k[3 * v];
        idx[((int64_t)kk[0] * n[1] + kk[1]) * n[2] + kk[2]] = v;
    }
    for (int d = 0; d < 3; d++) {
        p->mirror[d] = (int64_t *)malloc((size_t)p->nv * sizeof(int64_t));
        for (int64_t v = 0; v < p->nv; v++) {
            int32_t kk[3] = {p->k[3 * v], p->k[3 * v + 1], p->k[3 * v + 2]};
            kk[d] = n[d] - 1 - kk[d];
            p->mirror[d][v] = idx[((int64_t)kk[0] * n[1] + kk[1]) * n[2] + kk[2]];
        }
    }
    free(idx);
    p->f = with_f ? (double *)calloc((size_t)(p->ncells * p->nv), sizeof(double)) : NULL;
    p->finf = (double *)calloc((size_t)p->nv, sizeof(double));
    if ((with_f && !p->f) || !p->finf) { orc_destroy(p); return NULL; }
    double u0[3] = {0, 0, 0};
    orc_set_freestream(p, 1.0, u0, 1.0);
    return p;
}

orc_problem *orc_create(const orc_tree_spec *spec, const int n[3],
                        const double lo[3], const double hi[3])
{
    return create_grid(spec, n, lo, hi, 1);
}

orc_problem *orc_create_sparse(const orc_tree_spec *spec, const int n[3],
                               const double lo[3], const double hi[3])
{
    return create_grid(spec, n, lo, hi, 0);
}

void orc_destroy(orc_problem *p)
{
    if (!p) return;
    free(p->lv); free(p->cell_of_leaf); free(p->leaf_of_cell);
    free(p->fm); free(p->fp); free(p->fax); free(p->farea);
    free(p->cf_start); free(p->cf_list);
    free(p->bl); free(p->bother); free(p->bax); free(p->bside); free(p->bkind); free(p->barea);
    free(p->xi); free(p->k);
    for (int d = 0; d < 3; d++) free(p->mirror[d]);
    free(p->f); free(p->finf); free(p->lw);
    free(p->hs_start); free(p->hs_gam); free(p->hs_l); free(p->hs_m); free(p->hs_b);
    free(p);
}

int64_t orc_nleaves(const orc_problem *p) { return p->nleaves; }
int64_t orc_ncells(const orc_problem *p) { return p->ncells; }
int64_t orc_nv(const orc_problem *p) { return p->nv; }
int64_t orc_n_faces(const orc_problem *p) { return p->nf; }
int64_t orc_n_bfaces(const orc_problem *p) { return p->nbf; }

int orc_get_leaves(const orc_problem *p, uint64_t *keys, uint8_t *levels, uint8_t *solid)
{
    for (int64_t a = 0; a < p->nleaves; a++) {
        if (keys) keys[a] = p->lv[a].key;
        if (levels) levels[a] = (uint8_t)p->lv[a].lev;
        if (solid) solid[a] = p->lv[a].solid;
    }
    return 0;
}

int orc_cell_centres(const orc_problem *p, double *xyz, double *h)
{
    for (int64_t c = 0; c < p->ncells; c++) {
        const leaf_t *x = &p->lv[p->leaf_of_cell[c]];
        double hh = ldexp(1.0, -x->lev);
        for (int d = 0; d < 3; d++)
            xyz[3 * c + d] = d < p->spec.dim ? (x->i[d] + 0.5) * hh : 0.5;
        if (h) h[c] = hh;
    }
    return 0;
}

int orc_get_faces(const orc_problem *p, int64_t *minus, int64_t *plus,
                  uint8_t *axis, double *area)
{
    for (int64_t q = 0; q < p->nf; q++) {
        minus[q] = p->fm[q]; plus[q] = p->fp[q]; axis[q] = p->fax[q]; area[q] = p->farea[q];
    }
    return 0;
}

int orc_get_bfaces(const orc_problem *p, int64_t *leaf, uint8_t *axis,
                   uint8_t *side, uint8_t *kind, int64_t *other, double *area)
{
    for (int64_t q = 0; q < p->nbf; q++) {
        leaf[q] = p->bl[q]; axis[q] = p->bax[q]; side[q] = p->bside[q];
        kind[q] = p->bkind[q]; other[q] = p->bother[q]; area[q] = p->barea[q];
    }
    return 0;
}

int orc_set_freestream(orc_problem *p, double rho, const double u[3], double T)
{
    p->fs_rho = rho;
    p->fs_T = T;
    for (int d = 0; d < 3; d++) p->fs_u[d] = u[d];
    for (int64_t v = 0; v < p->nv; v++) p->finf[v] = maxwellian(rho, u, T, &p->xi[3 * v]);
    return 0;
}

int orc_init_maxwellian(orc_problem *p, int nmix, const double *w,
                        const double *rho, const double *u, const double *T)
{
    if (!p->f) return -1; /* a problem without f storage */
    return orc_maxwellian_rows(p, p->ncells, nmix, w, rho, u, T, p->f);
}

int orc_get_f(const orc_problem *p, double *f)
{
    if (!p->f) return -1; /* a problem without f storage */
    memcpy(f, p->f, (size_t)(p->ncells * p->nv) * sizeof(double));
    return 0;
}

int orc_set_f(orc_problem *p, const double *f)
{
    if (!p->f) return -1; /* a problem without f storage */
    memcpy(p->f, f, (size_t)(p->ncells * p->nv) * sizeof(double));
    return 0;
}

/* dt = CFL * h_min / max_i sum_{d < dim} |xi_{d,i}| */
double orc_dt_cfl(const orc_problem *p, double cfl)
{
    int maxlev = -1;
    for (int64_t c = 0; c < p->ncells; c++) {
        int l = p->lv[p->leaf_of_cell[c]].lev;
        if (l > maxlev) maxlev = l;
    }
    double smax = 0.0;
    for (int64_t v = 0; v < p->nv; v++) {
        double s = 0.0;
        for (int d = 0; d < p->spec.dim; d++) s += fabs(p->xi[3 * v + d]);
        if (s > smax) smax = s;
    }
    return cfl * ldexp(1.0, -maxlev) / smax;
}

/* ------------------------------------------------------------------------ */
/* Transport, Eq. 2 written as a sum of upwind face fluxes:
 *   f*_j = f_j - (dt / V_j) sum_{faces of j} (xi . n_out) A f_upwind
 * The upwind value is the cell on the side the velocity comes from; at a
 * domain side it is the ghost value (inflow: freestream Maxwellian;
 * outflow: the cell's own value; specular wall: the cell's value at the
 * reflected velocity). */
/* f* of cell c into out; row(ctx, k) gives the f row of cell k */
typedef const double *(*row_fn)(const orc_problem *p, const void *ctx, int64_t k);

static void transport_cell(const orc_problem *p, int64_t c, row_fn row, const void *ctx, double dt, double *out)
{
    int dim = p->spec.dim;
    int64_t nv = p->nv;
    const double *own = row(p, ctx, c);
    double V = ldexp(1.0, -p->lv[p->leaf_of_cell[c]].lev * dim);
    for (int64_t v = 0; v < nv; v++) out[v] = own[v];
    for (int64_t e = p->cf_start[c]; e < p->cf_start[c + 1]; e++) {
        int64_t q = p->cf_list[e];
        if (q >= 0) {
            /* interior face: flux from minus to plus along +axis */
            int d = p->fax[q];
            int64_t a = p->cell_of_leaf[p->fm[q]], b = p->cell_of_leaf[p->fp[q]];
            double sgn = (a == c) ? 1.0 : -1.0; /* outward normal of this cell */
            const double *fa = row(p, ctx, a), *fb = row(p, ctx, b);
            for (int64_t v = 0; v < nv; v++) {
                double x = p->xi[3 * v + d];
                double up = x > 0.0 ? fa[v] : fb[v];
                double flux = x * p->farea[q] * up;
                out[v] -= sgn * dt * flux / V;
            }
        } else {
            q = -1 - q;
            int d = p->bax[q];
            for (int64_t v = 0; v < nv; v++) {
                double xn = (p->bside[q] ? 1.0 : -1.0) * p->xi[3 * v + d];
                double up;
                if (xn > 0.0) up = own[v];
                else if (p->bkind[q] == ORC_BC_INFLOW) up = p->finf[v];
                else if (p->bkind[q] == ORC_BC_WALL) up = own[p->mirror[d][v]];
                else up = own[v];
                out[v] -= dt * xn * p->barea[q] * up / V;
            }
        }
    }
}

static const double *row_dense(const orc_problem *p, const void *ctx, int64_t k)
{
    (void)ctx;
    return &p->f[k * p->nv];
}

int orc_transport(orc_problem *p, double dt)
{
    if (!p->f) return -1; /* a problem without f storage */
    int64_t nv = p->nv;
    double *fs = (double *)malloc((size_t)(p->ncells * nv) * sizeof(double));
    if (!fs) return -1;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t c = 0; c < p->ncells; c++) transport_cell(p, c, row_dense, NULL, dt, &fs[c * nv]);
    free(p->f);
    p->f = fs;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Moments: rho = sum f dV, rho u = sum xi f dV, E = sum |xi|^2/2 f dV,
 * T = (2E/rho - |u|^2)/3 (velocities in thermal units). */
static void cell_moments(const orc_problem *p, const double *f, double *rho,
                         double u[3], double *T)
{
    double s0 = 0.0, s1[3] = {0, 0, 0}, s2 = 0.0;
    for (int64_t v = 0; v < p->nv; v++) {
        const double *x = &p->xi[3 * v];
        s0 += f[v];
        for (int d = 0; d < 3; d++) s1[d] += x[d] * f[v];
        s2 += (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) * f[v];
    }
    *rho = s0 * p->dV;
    double uu = 0.0;
    for (int d = 0; d < 3; d++) { u[d] = s1[d] / s0; uu += u[d] * u[d]; }
    *T = (s2 / s0 - uu) / 3.0;
}

int orc_moments(const orc_problem *p, double *rho, double *u, double *T)
{
    if (!p->f) return -1; /* a problem without f storage */
    for (int64_t c = 0; c < p->ncells; c++)
        cell_moments(p, &p->f[c * p->nv], &rho[c], &u[3 * c], &T[c]);
    return 0;
}

int orc_totals(const orc_problem *p, double out[5])
{
    if (!p->f) return -1; /* a problem without f storage */
    for (int r = 0; r < 5; r++) out[r] = 0.0;
    int dim = p->spec.dim;
    for (int64_t c = 0; c < p->ncells; c++) {
        double V = ldexp(1.0, -p->lv[p->leaf_of_cell[c]].lev * dim);
        for (int64_t v = 0; v < p->nv; v++) {
            const double *x = &p->xi[3 * v];
            double fv = p->f[c * p->nv + v] * p->dV * V;
            out[0] += fv;
            out[1] += x[0] * fv;
            out[2] += x[1] * fv;
            out[3] += x[2] * fv;
            out[4] += (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]) * fv;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */

int orc_solve(int n, double *A, double *b, double *x)
{
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (!(fabs(A[piv * n + c]) > 0.0) || !isfinite(A[piv * n + c])) return -1;
        if (piv != c) {
            for (int q = 0; q < n; q++) { double t = A[c * n + q]; A[c * n + q] = A[piv * n + q]; A[piv * n + q] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; r++) {
            double m = A[r * n + c] / A[c * n + c];
            for (int q = c; q < n; q++) A[r * n + q] -= m * A[c * n + q];
            b[r] -= m * b[c];
        }
    }
    for (int r = n - 1; r >= 0; r--) {
        double s = b[r];
        for (int q = r + 1; q < n; q++) s -= A[r * n + q] * x[q];
        x[r] = s / A[r * n + r];
        if (!isfinite(x[r])) return -1;
    }
    return 0;
}

static void psi5(const double *x, double ps[5])
{
    ps[0] = 1.0; ps[1] = x[0]; ps[2] = x[1]; ps[3] = x[2];
    ps[4] = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
}

/* Conservative BGK: the discrete Maxwellian of the cell's moments times the
 * polynomial 1 + d0 + d.xi + d2 |xi|^2 (the correction form of Eq. 6) whose
 * five coefficients make its discrete moments equal those of f; then
 * f <- f + dt nu (M~ - f), nu = sqrt(8/pi) rho sqrt(T) / Kn. */
/* the update of one cell's f (in place); q (may be NULL) gets the term */
static int bgk_cell(const orc_problem *p, double *f, double dt, double kn, double *q)
{
    int64_t nv = p->nv;
    double rho, u[3], T;
    cell_moments(p, f, &rho, u, &T);
    double *M = (double *)malloc((size_t)nv * sizeof(double));
    double A[25] = {0}, rhs[5] = {0}, d[5];
    for (int64_t v = 0; v < nv; v++) {
        double ps[5];
        psi5(&p->xi[3 * v], ps);
        M[v] = maxwellian(rho, u, T, &p->xi[3 * v]);
        for (int r = 0; r < 5; r++) {
            for (int s = 0; s < 5; s++) A[r * 5 + s] += ps[r] * ps[s] * M[v] * p->dV;
            rhs[r] += ps[r] * (f[v] - M[v]) * p->dV;
        }
    }
    if (!(rho > 0.0) || !(T > 0.0) || orc_solve(5, A, rhs, d)) { free(M); return -1; }
    double nu = sqrt(8.0 / M_PI) * rho * sqrt(T) / kn;
    for (int64_t v = 0; v < nv; v++) {
        double ps[5];
        psi5(&p->xi[3 * v], ps);
        double P = 1.0;
        for (int r = 0; r < 5; r++) P += d[r] * ps[r];
        double Q = nu * (M[v] * P - f[v]);
        if (q) q[v] = Q;
        f[v] += dt * Q;
    }
    free(M);
    return 0;
}

int orc_bgk(orc_problem *p, double dt, double kn, double *q)
{
    if (!p->f) return -1; /* a problem without f storage */
    int64_t nv = p->nv;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
    for (int64_t c = 0; c < p->ncells; c++)
        if (bgk_cell(p, &p->f[c * nv], dt, kn, q ? &q[c * nv] : NULL)) err = 1;
    return err ? -1 : 0;
}

/* ---- one step of selected cells, for trees whose f does not fit in host
 * memory: the cells a step of `cells` reads, their f rows supplied by the
 * caller, and the stepped rows (transport, Eq. 2, then conservative BGK). */
static int cmp_i64(const void *a, const void *b)
{
    const int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int64_t orc_step_inputs(const orc_problem *p, int64_t n, const int64_t *cells, int64_t *out)
{
    int64_t cap = 0;
    for (int64_t i = 0; i < n; i++) {
        if (cells[i] < 0 || cells[i] >= p->ncells) return -1;
        cap += 1 + 2 * (p->cf_start[cells[i] + 1] - p->cf_start[cells[i]]);
    }
    int64_t *t = (int64_t *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int64_t));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++) {
        const int64_t c = cells[i];
        t[m++] = c;
        for (int64_t e = p->cf_start[c]; e < p->cf_start[c + 1]; e++) {
            const int64_t q = p->cf_list[e];
            if (q >= 0) {
                t[m++] = p->cell_of_leaf[p->fm[q]];
                t[m++] = p->cell_of_leaf[p->fp[q]];
            }
        }
    }
    qsort(t, (size_t)m, sizeof(int64_t), cmp_i64);
    int64_t k = 0;
    for (int64_t i = 0; i < m; i++)
        if (k == 0 || t[i] != t[k - 1]) t[k++] = t[i];
    if (out) memcpy(out, t, (size_t)k * sizeof(int64_t));
    free(t);
    return k;
}

int orc_maxwellian_rows(const orc_problem *p, int64_t nrows, int nmix, const double *w, const double *rho,
                        const double *u, const double *T, double *out)
{
    for (int64_t c = 0; c < nrows; c++)
        for (int64_t v = 0; v < p->nv; v++) {
            double s = 0.0;
            for (int m = 0; m < nmix; m++) {
                int64_t q = c * nmix + m;
                s += w[q] * maxwellian(rho[q], &u[3 * q], T[q], &p->xi[3 * v]);
            }
            out[c * p->nv + v] = s;
        }
    return 0;
}

typedef struct {
    int64_t n;
    const int64_t *cells;
    const double *rows;
} row_table;

static const double *row_sparse(const orc_problem *p, const void *ctx, int64_t k)
{
    const row_table *t = (const row_table *)ctx;
    int64_t lo = 0, hi = t->n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi) / 2;
        if (t->cells[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    return t->n > 0 && t->cells[lo] == k ? &t->rows[lo * p->nv] : NULL;
}


/* Entropic BGK (the discrete entropic equilibrium, a reading of the
 * correction of Sec. 3.2 that keeps the H-theorem exact): the target is
 * E = exp(a . psi) with psi = (1, xi, |xi|^2), the five multipliers a chosen
 * so that sum psi E dV equals sum psi f dV; E minimises sum E ln E dV under
 * those moments.  Newton's method from the continuous Maxwellian's
 * multipliers (a0 = ln(rho (2 pi T)^(-3/2)) - |u|^2/(2T), a_d = u_d/T,
 * a4 = -1/(2T)), every sum over all nodes, until each moment defect is below
 * 1e-14 of its scale.  Then f <- f + dt nu (E - f), nu as for BGK. */
int orc_bgk_entropic(orc_problem *p, double dt, double kn, double *q)
{
    if (!p->f) return -1; /* a problem without f storage */
    int64_t nv = p->nv;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : err)
    for (int64_t c = 0; c < p->ncells; c++) {
        double *f = &p->f[c * nv];
        double rho, u[3], T;
        cell_moments(p, f, &rho, u, &T);
        if (!(rho > 0.0) || !(T > 0.0)) { err = 1; continue; }
        double m[5] = {0}, scale[5] = {0};
        for (int64_t v = 0; v < nv; v++) {
            double ps[5];
            psi5(&p->xi[3 * v], ps);
            for (int r = 0; r < 5; r++) {
                m[r] += ps[r] * f[v] * p->dV;
                scale[r] += fabs(ps[r]) * fabs(f[v]) * p->dV;
            }
        }
        double a[5];
        const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        a[0] = log(rho / pow(2.0 * M_PI * T, 1.5)) - u2 / (2.0 * T);
        for (int d = 0; d < 3; d++) a[1 + d] = u[d] / T;
        a[4] = -1.0 / (2.0 * T);
        int ok = 0;
        for (int it = 0; it < 50 && !ok; it++) {
            double G[5] = {0}, J[25] = {0}, da[5];
            for (int64_t v = 0; v < nv; v++) {
                double ps[5];
                psi5(&p->xi[3 * v], ps);
                double e = 0.0;
                for (int r = 0; r < 5; r++) e += a[r] * ps[r];
                e = exp(e) * p->dV;
                for (int r = 0; r < 5; r++) {
                    G[r] += ps[r] * e;
                    for (int t = 0; t < 5; t++) J[r * 5 + t] += ps[r] * ps[t] * e;
                }
            }
            double worst = 0.0;
            for (int r = 0; r < 5; r++) {
                G[r] -= m[r];
                worst = fmax(worst, fabs(G[r]) / scale[r]);
            }
            if (worst < 1e-14) { ok = 1; break; }
            if (orc_solve(5, J, G, da)) break;
            for (int r = 0; r < 5; r++) a[r] -= da[r];
        }
        if (!ok) { err = 1; continue; }
        double nu = sqrt(8.0 / M_PI) * rho * sqrt(T) / kn;
        for (int64_t v = 0; v < nv; v++) {
            double ps[5];
            psi5(&p->xi[3 * v], ps);
            double e = 0.0;
            for (int r = 0; r < 5; r++) e += a[r] * ps[r];
            double Q = nu * (exp(e) - f[v]);
            if (q) q[c * nv + v] = Q;
            f[v] += dt * Q;
        }
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Hard-sphere trials.  For node i and trial k the stream index is i*M + k
 * and draws 3s, 3s+1, 3s+2 give the partner gamma (uniform over the nodes)
 * and the unit vector omega (z = 2u - 1, phi = 2 pi u').  The post-collision
 * pair xi' = c + |g| omega / 2, xi'_* = c - |g| omega / 2 (c the mean of xi_i
 * and xi_gamma) is mapped to its nearest nodes l, m; a trial whose l or m
 * falls outside the grid is dropped.  With M the number of trials drawn
 * (dropped ones included: they stand for partners in the tails, where f is
 * negligible), b = c = Nv dV |g| / (sqrt(2) M), the Monte-Carlo weights of
 * I = 1/(4 sqrt(2) pi) int int (f'f'_* - f f_*) |g| dOmega dxi_*. */
static int nearest_node(const orc_problem *p, const double x[3], int32_t kk[3])
{
    for (int d = 0; d < 3; d++) {
        double t = (x[d] - p->lo[d]) / p->h[d] - 0.5;
        double r = round(t);
        if (!(r >= 0.0) || r > (double)(p->n[d] - 1)) return 0;
        kk[d] = (int32_t)r;
    }
    return 1;
}

/* Korobov rank-1 lattice of M points in [0,1)^5 (the quadrature family of
 * the paper's Ref. [5] for the collision integral): point k is
 * frac(k (1, a, a^2, a^3, a^4 mod M) / M).  The multiplier a is the odd
 * integer in [1, M) that maximises the smallest distance between two lattice
 * points on the unit torus (squared distances in units of 1/M^2, integers),
 * the smallest such a on ties. */
int64_t orc_korobov_a(int64_t M)
{
    int64_t best = 1, bestd = -1;
    for (int64_t a = 1; a < M; a += 2) {
        int64_t z[5];
        z[0] = 1;
        for (int j = 1; j < 5; j++) z[j] = (z[j - 1] * a) % M;
        int64_t dmin = INT64_MAX;
        for (int64_t k = 1; k < M && dmin > bestd; k++) {
            int64_t d2 = 0;
            for (int j = 0; j < 5; j++) {
                int64_t r = (k * z[j]) % M;
                if (M - r < r) r = M - r;
                d2 += r * r;
            }
            if (d2 < dmin) dmin = d2;
        }
        if (dmin > bestd) {
            bestd = dmin;
            best = a;
        }
    }
    return best;
}

/* The uniform numbers of trial k of node i.  Random trials: three SplitMix64
 * draws 3s, 3s+1, 3s+2 with s = i M + k (u[3], u[4] unused).  Lattice
 * trials: the five coordinates of Korobov point k, shifted per node by the
 * SplitMix64 draws 5i .. 5i+4 modulo 1 (a random shift of the lattice for
 * every node). */
static void trial_uniforms(int lattice, uint64_t seed, int64_t i, int64_t k, int64_t M, const int64_t z[5],
                           double u[5])
{
    if (lattice) {
        for (int j = 0; j < 5; j++) {
            double t = (double)((k * z[j]) % M) / (double)M + unif53(seed, 5 * (uint64_t)i + (uint64_t)j);
            if (t >= 1.0) t -= 1.0;
            u[j] = t;
        }
    } else {
        const uint64_t s = (uint64_t)i * (uint64_t)M + (uint64_t)k;
        for (int j = 0; j < 3; j++) u[j] = unif53(seed, 3 * s + (uint64_t)j);
        u[3] = u[4] = 0.0;
    }
}

static int hs_tables(orc_problem *p, int trials, uint64_t seed, int lattice)
{
    int64_t nv = p->nv;
    int64_t *idx = (int64_t *)malloc((size_t)nv * sizeof(int64_t));
    for (int64_t v = 0; v < nv; v++) {
        const int32_t *kk = &p->k[3 * v];
        idx[((int64_t)kk[0] * p->n[1] + kk[1]) * p->n[2] + kk[2]] = v;
    }
    free(p->hs_start); free(p->hs_gam); free(p->hs_l); free(p->hs_m); free(p->hs_b);
    int64_t cap = nv * trials;
    p->hs_start = (int64_t *)malloc((size_t)(nv + 1) * sizeof(int64_t));
    p->hs_gam = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    p->hs_l = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    p->hs_m = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
    p->hs_b = (double *)malloc((size_t)cap * sizeof(double));
    int64_t z[5] = {1, 1, 1, 1, 1};
    if (lattice) {
        const int64_t a = orc_korobov_a(trials);
        for (int j = 1; j < 5; j++) z[j] = (z[j - 1] * a) % trials;
    }
    int64_t nk = 0, disc = 0;
    for (int64_t i = 0; i < nv; i++) {
        p->hs_start[i] = nk;
        const double *xa = &p->xi[3 * i];
        for (int k = 0; k < trials; k++) {
            double u[5];
            trial_uniforms(lattice, seed, i, k, trials, z, u);
            /* partner: uniform over the nodes, as a storage index (random) or
             * as the node of axis indices floor(u_d n_d) (lattice: smooth in
             * the lattice coordinates); unit vector omega from the last two */
            int64_t gam;
            double uz, uphi;
            if (lattice) {
                int64_t kk[3];
                for (int d = 0; d < 3; d++) {
                    kk[d] = (int64_t)(u[d] * (double)p->n[d]);
                    if (kk[d] > p->n[d] - 1) kk[d] = p->n[d] - 1;
                }
                gam = idx[(kk[0] * p->n[1] + kk[1]) * p->n[2] + kk[2]];
                uz = u[3];
                uphi = u[4];
            } else {
                gam = (int64_t)(u[0] * (double)nv);
                uz = u[1];
                uphi = u[2];
            }
            const double *xb = &p->xi[3 * gam];
            double g2 = 0.0;
            for (int d = 0; d < 3; d++) g2 += (xa[d] - xb[d]) * (xa[d] - xb[d]);
            double gn = sqrt(g2);
            double zc = 2.0 * uz - 1.0, phi = 2.0 * M_PI * uphi;
            double st = sqrt(fmax(0.0, 1.0 - zc * zc));
            double w[3] = {st * cos(phi), st * sin(phi), zc};
            double xp[3], xq[3];
            for (int d = 0; d < 3; d++) {
                double c = 0.5 * (xa[d] + xb[d]);
                xp[d] = c + 0.5 * gn * w[d];
                xq[d] = c - 0.5 * gn * w[d];
            }
            int32_t kp[3], kq[3];
            if (!nearest_node(p, xp, kp) || !nearest_node(p, xq, kq)) { disc++; continue; }
            p->hs_gam[nk] = (int32_t)gam;
            p->hs_l[nk] = (int32_t)idx[((int64_t)kp[0] * p->n[1] + kp[1]) * p->n[2] + kp[2]];
            p->hs_m[nk] = (int32_t)idx[((int64_t)kq[0] * p->n[1] + kq[1]) * p->n[2] + kq[2]];
            p->hs_b[nk] = gn;
            nk++;
        }
        for (int64_t q = p->hs_start[i]; q < nk; q++)
            p->hs_b[q] = (double)nv * p->dV * p->hs_b[q] / (sqrt(2.0) * (double)trials);
    }
    p->hs_start[nv] = nk;
    p->hs_nkept = nk;
    p->hs_discarded = disc;
    p->hs_trials = trials;
    free(idx);
    return 0;
}

int orc_hs_tables(orc_problem *p, int trials, uint64_t seed) { return hs_tables(p, trials, seed, 0); }

void orc_trial_uniforms(int lattice, uint64_t seed, int64_t i, int64_t k, int64_t M, double *u)
{
    int64_t z[5] = {1, 1, 1, 1, 1};
    if (lattice) {
        const int64_t a = orc_korobov_a(M);
        for (int j = 1; j < 5; j++) z[j] = (z[j - 1] * a) % M;
    }
    trial_uniforms(lattice, seed, i, k, M, z, u);
}

int orc_hs_tables_lattice(orc_problem *p, int trials, uint64_t seed)
{
    if (trials < 2) return -1;
    return hs_tables(p, trials, seed, 1);
}

int64_t orc_hs_nkept(const orc_problem *p) { return p->hs_nkept; }

int orc_hs_get_tables(const orc_problem *p, int64_t *start, int32_t *gam,
                      int32_t *l, int32_t *m, double *b, int64_t *discarded)
{
    if (!p->hs_start) return -1;
    memcpy(start, p->hs_start, (size_t)(p->nv + 1) * sizeof(int64_t));
    memcpy(gam, p->hs_gam, (size_t)p->hs_nkept * sizeof(int32_t));
    memcpy(l, p->hs_l, (size_t)p->hs_nkept * sizeof(int32_t));
    memcpy(m, p->hs_m, (size_t)p->hs_nkept * sizeof(int32_t));
    memcpy(b, p->hs_b, (size_t)p->hs_nkept * sizeof(double));
    *discarded = p->hs_discarded;
    return 0;
}

/* Eqs. 4-6: B_i = sum_k b f_gamma, C_i = sum_k c f_l f_m (b = c),
 * I_i = -f_i P_i B_i + C_i with P = 1 + d0 + d.xi + d2 |xi|^2 chosen so that
 * sum_i psi_r I_i dV = 0 for psi = (1, xi, |xi|^2); then f <- f + dt/Kn I. */
/* the hard-sphere update of one cell's f (in place); q, Bout, Cout (each may
 * be NULL) get I, B and C of the cell */
static int hs_cell(const orc_problem *p, double *f, double dt, double kn, double *q, double *Bout, double *Cout)
{
    int64_t nv = p->nv;
    double *B = (double *)malloc((size_t)nv * sizeof(double));
    double *C = (double *)malloc((size_t)nv * sizeof(double));
    for (int64_t i = 0; i < nv; i++) {
        double sb = 0.0, sc = 0.0;
        for (int64_t t = p->hs_start[i]; t < p->hs_start[i + 1]; t++) {
            sb += p->hs_b[t] * f[p->hs_gam[t]];
            sc += p->hs_b[t] * f[p->hs_l[t]] * f[p->hs_m[t]];
        }
        B[i] = sb;
        C[i] = sc;
    }
    double A[25] = {0}, rhs[5] = {0}, d[5];
    for (int64_t i = 0; i < nv; i++) {
        double ps[5];
        psi5(&p->xi[3 * i], ps);
        for (int r = 0; r < 5; r++) {
            for (int s = 0; s < 5; s++) A[r * 5 + s] += ps[r] * ps[s] * f[i] * B[i] * p->dV;
            rhs[r] += ps[r] * (C[i] - f[i] * B[i]) * p->dV;
        }
    }
    if (orc_solve(5, A, rhs, d)) { free(B); free(C); return -1; }
    for (int64_t i = 0; i < nv; i++) {
        double ps[5];
        psi5(&p->xi[3 * i], ps);
        double P = 1.0;
        for (int r = 0; r < 5; r++) P += d[r] * ps[r];
        double I = -f[i] * P * B[i] + C[i];
        if (q) q[i] = I;
        if (Bout) Bout[i] = B[i];
        if (Cout) Cout[i] = C[i];
        f[i] += dt / kn * I;
    }
    free(B);
    free(C);
    return 0;
}

int orc_hs_collide(orc_problem *p, double dt, double kn, double *q,
                   double *Bout, double *Cout)
{
    if (!p->f) return -1; /* a problem without f storage */
    if (!p->hs_start) return -1;
    int64_t nv = p->nv;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : err)
    for (int64_t c = 0; c < p->ncells; c++)
        if (hs_cell(p, &p->f[c * nv], dt, kn, q ? &q[c * nv] : NULL, Bout ? &Bout[c * nv] : NULL,
                    Cout ? &Cout[c * nv] : NULL))
            err = 1;
    return err ? -1 : 0;
}

int orc_step_cells(const orc_problem *p, int64_t n, const int64_t *cells, int64_t ninp, const int64_t *inputs,
                   const double *fin, double dt, int coll, double kn, double *out)
{
    /* coll as in orc_step: 1 BGK, 2 hard sphere */
    if (coll != 1 && coll != 2) return -1;
    if (coll == 2 && !p->hs_start) return -1;
    row_table t = {ninp, inputs, fin};
    for (int64_t i = 0; i < n; i++) {
        /* every row the cell reads must be supplied */
        if (cells[i] < 0 || cells[i] >= p->ncells || !row_sparse(p, &t, cells[i])) return -1;
        for (int64_t e = p->cf_start[cells[i]]; e < p->cf_start[cells[i] + 1]; e++) {
            const int64_t q = p->cf_list[e];
            if (q >= 0 && (!row_sparse(p, &t, p->cell_of_leaf[p->fm[q]]) || !row_sparse(p, &t, p->cell_of_leaf[p->fp[q]])))
                return -1;
        }
    }
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t i = 0; i < n; i++) {
        double *o = &out[i * p->nv];
        transport_cell(p, cells[i], row_sparse, &t, dt, o);
        const int rc = coll == 1 ? bgk_cell(p, o, dt, kn, NULL) : hs_cell(p, o, dt, kn, NULL, NULL, NULL);
        if (rc) err = 1;
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Lie splitting: transport, then the collision update on f*. */
/* ------------------------------------------------------------------------ */
/* Lattice Boltzmann on the tree (Sec. 4): the LBM module is the DVM solver on
 * a minimal velocity set, D2Q9 (3x3), D3Q19 or D3Q27 (3x3x3), with lattice
 * weights w_i and lattice speed of sound c_s = 1/sqrt(3).  Transport is the
 * same finite-volume upwind scheme (orc_transport, Eq. 2, finite-volume LBM
 * as in the paper's Ref. [44]); a velocity component of 0 carries no flux.
 * Collision is the BGK form I_i = -(f_i - feq_i)/tau with the second-order
 * equilibrium
 *   feq_i = w_i rho (1 + c_i.u/c_s^2 + (c_i.u)^2/(2 c_s^4) - |u|^2/(2 c_s^2)),
 * rho = sum_i f_i, rho u = sum_i c_i f_i.  Velocity order: increasing |c|^2,
 * ties lexicographic in (c_x, c_y, c_z) with -1 < 0 < 1.  Weights by |c|^2:
 * D2Q9 4/9, 1/9, 1/36; D3Q19 1/3, 1/18, 1/36; D3Q27 8/27, 2/27, 1/54, 1/216
 * (the values fixed by 4th-order isotropy of each set).  dV = 1, so the DVM
 * moments routine returns rho and u of the lattice. */
static int lattice_set(int lattice, int dim, double *c, double *w)
{
    static const double w9[3] = {4.0 / 9, 1.0 / 9, 1.0 / 36};
    static const double w19[3] = {1.0 / 3, 1.0 / 18, 1.0 / 36};
    static const double w27[4] = {8.0 / 27, 2.0 / 27, 1.0 / 54, 1.0 / 216};
    int q = 0;
    for (int r = 0; r <= 3; r++)
        for (int x = -1; x <= 1; x++)
            for (int y = -1; y <= 1; y++)
                for (int z = -1; z <= 1; z++) {
                    int r2 = x * x + y * y + z * z;
                    if (r2 != r) continue;
                    double wt;
                    if (lattice == ORC_D2Q9) {
                        if (z != 0) continue;
                        wt = w9[r2];
                    } else if (lattice == ORC_D3Q19) {
                        if (r2 == 3) continue;
                        wt = w19[r2];
                    } else {
                        wt = w27[r2];
                    }
                    if (c) { c[3 * q] = x; c[3 * q + 1] = y; c[3 * q + 2] = z; }
                    if (w) w[q] = wt;
                    q++;
                }
    (void)dim;
    return q;
}

int orc_lattice_q(int lattice)
{
    if (lattice != ORC_D2Q9 && lattice != ORC_D3Q19 && lattice != ORC_D3Q27) return -1;
    return lattice_set(lattice, 0, NULL, NULL);
}

int orc_lattice(int lattice, double *c, double *w)
{
    if (orc_lattice_q(lattice) < 0) return -1;
    lattice_set(lattice, 0, c, w);
    return 0;
}

orc_problem *orc_create_lattice(const orc_tree_spec *spec, int lattice)
{
    int Q = orc_lattice_q(lattice);
    if (Q < 0 || (lattice == ORC_D2Q9) != (spec->dim == 2)) return NULL;
    orc_problem *p = create_tree(spec);
    if (!p) return NULL;
    p->lattice = lattice;
    p->nv = Q;
    p->dV = 1.0;
    for (int d = 0; d < 3; d++) { p->n[d] = 3; p->lo[d] = -1.5; p->hi[d] = 1.5; p->h[d] = 1.0; }
    p->xi = (double *)malloc((size_t)Q * 3 * sizeof(double));
    p->lw = (double *)malloc((size_t)Q * sizeof(double));
    lattice_set(lattice, spec->dim, p->xi, p->lw);
    /* mirror maps: the velocity with component d negated (a set member) */
    for (int d = 0; d < 3; d++) {
        p->mirror[d] = (int64_t *)malloc((size_t)Q * sizeof(int64_t));
        for (int v = 0; v < Q; v++) {
            double r[3] = {p->xi[3 * v], p->xi[3 * v + 1], p->xi[3 * v + 2]};
            r[d] = -r[d];
            p->mirror[d][v] = -1;
            for (int t = 0; t < Q; t++)
                if (p->xi[3 * t] == r[0] && p->xi[3 * t + 1] == r[1] && p->xi[3 * t + 2] == r[2])
                    p->mirror[d][v] = t;
        }
    }
    p->f = (double *)calloc((size_t)(p->ncells * Q), sizeof(double));
    p->finf = (double *)calloc((size_t)Q, sizeof(double));
    if (!p->f || !p->finf) { orc_destroy(p); return NULL; }
    double u0[3] = {0, 0, 0};
    orc_lbm_set_inflow(p, 1.0, u0);
    return p;
}

int orc_lbm_feq(const orc_problem *p, double rho, const double u[3], double *feq)
{
    if (!p->lattice) return -1;
    const double cs2 = 1.0 / 3.0;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int64_t v = 0; v < p->nv; v++) {
        const double *c = &p->xi[3 * v];
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        feq[v] = p->lw[v] * rho * (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));
    }
    return 0;
}

int orc_lbm_set_inflow(orc_problem *p, double rho, const double u[3])
{
    p->fs_rho = rho;
    for (int d = 0; d < 3; d++) p->fs_u[d] = u[d];
    return orc_lbm_feq(p, rho, u, p->finf);
}

int orc_lbm_init(orc_problem *p, const double *rho, const double *u)
{
    for (int64_t c = 0; c < p->ncells; c++)
        if (orc_lbm_feq(p, rho[c], &u[3 * c], &p->f[c * p->nv])) return -1;
    return 0;
}

/* rho and u of every cell: rho = sum f, u = sum c f / rho */
int orc_lbm_moments(const orc_problem *p, double *rho, double *u)
{
    for (int64_t c = 0; c < p->ncells; c++) {
        const double *f = &p->f[c * p->nv];
        double s0 = 0.0, s1[3] = {0, 0, 0};
        for (int64_t v = 0; v < p->nv; v++) {
            s0 += f[v];
            for (int d = 0; d < 3; d++) s1[d] += p->xi[3 * v + d] * f[v];
        }
        rho[c] = s0;
        for (int d = 0; d < 3; d++) u[3 * c + d] = s1[d] / s0;
    }
    return 0;
}

/* f <- f - (dt/tau) (f - feq(rho(f), u(f))) in every cell; -1 if a cell has
 * rho <= 0 or non-finite moments */
int orc_lbm_collide(orc_problem *p, double dt, double tau)
{
    int err = 0;
    const double om = dt / tau;
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int64_t c = 0; c < p->ncells; c++) {
        double *f = &p->f[c * p->nv];
        double rho = 0.0, j[3] = {0, 0, 0};
        for (int64_t v = 0; v < p->nv; v++) {
            rho += f[v];
            for (int d = 0; d < 3; d++) j[d] += p->xi[3 * v + d] * f[v];
        }
        if (!(rho > 0.0) || !isfinite(j[0] + j[1] + j[2])) { err = 1; continue; }
        double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
        double feq[27];
        orc_lbm_feq(p, rho, u, feq);
        for (int64_t v = 0; v < p->nv; v++) f[v] -= om * (f[v] - feq[v]);
    }
    return err ? -1 : 0;
}

int orc_lbm_step(orc_problem *p, int nsteps, double dt, double tau)
{
    if (!p->lattice) return -1;
    for (int s = 0; s < nsteps; s++) {
        if (orc_transport(p, dt)) return -1;
        if (orc_lbm_collide(p, dt, tau)) return -2;
    }
    return 0;
}

int orc_step(orc_problem *p, int nsteps, double dt, int coll, double kn)
{
    if (!p->f) return -1; /* a problem without f storage */
    for (int s = 0; s < nsteps; s++) {
        if (orc_transport(p, dt)) return -1;
        if (coll == 1 && orc_bgk(p, dt, kn, NULL)) return -2;
        if (coll == 2 && orc_hs_collide(p, dt, kn, NULL, NULL, NULL)) return -3;
        if (coll == 4 && orc_bgk_entropic(p, dt, kn, NULL)) return -4;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Local Knudsen number.  The gradient of a moment q at cell j is the
 * weighted least-squares fit over its fluid face neighbours k,
 *   min_g sum_k w_k (q_k - q_j - g.(x_k - x_j))^2,  w_k = A_k / |x_k - x_j|^2,
 * which is exact for linear fields on any 2:1 stencil (a component with no
 * neighbour spread, e.g. a cell walled in along that axis, is set to 0). */
/* local Kn of cell c from the moments (rho, u [3 per cell], T) and centres
 * xc [3 per cell] of the cell and its fluid face neighbours */
static double kn_cell(const orc_problem *p, int64_t c, double kn, const double *rho, const double *u, const double *T,
                      const double *xc)
{
    int dim = p->spec.dim;
    double q[5] = {rho[c], T[c], u[3 * c], u[3 * c + 1], u[3 * c + 2]};
    double N[9] = {0}, R[5][3] = {{0}};
    for (int64_t e = p->cf_start[c]; e < p->cf_start[c + 1]; e++) {
        int64_t f = p->cf_list[e];
        if (f < 0) continue; /* boundary face: no fluid neighbour */
        int64_t a = p->cell_of_leaf[p->fm[f]], b = p->cell_of_leaf[p->fp[f]];
        int64_t nb = (a == c) ? b : a;
        double d[3] = {0, 0, 0}, d2 = 0.0;
        for (int k = 0; k < dim; k++) {
            d[k] = xc[3 * nb + k] - xc[3 * c + k];
            if (p->spec.bc[2 * k] == ORC_BC_PERIODIC) {
                if (d[k] > 0.5) d[k] -= 1.0;
                if (d[k] < -0.5) d[k] += 1.0;
            }
            d2 += d[k] * d[k];
        }
        double w = p->farea[f] / d2;
        double qn[5] = {rho[nb], T[nb], u[3 * nb], u[3 * nb + 1], u[3 * nb + 2]};
        for (int r = 0; r < dim; r++) {
            for (int k = 0; k < dim; k++) N[r * 3 + k] += w * d[r] * d[k];
            for (int m = 0; m < 5; m++) R[m][r] += w * d[r] * (qn[m] - q[m]);
        }
    }
    double grad[5][3] = {{0}};
    for (int m = 0; m < 5; m++) {
        double A[9], bb[3], g[3] = {0, 0, 0};
        for (int r = 0; r < dim; r++) {
            for (int k = 0; k < dim; k++) A[r * dim + k] = N[r * 3 + k];
            bb[r] = R[m][r];
        }
        if (orc_solve(dim, A, bb, g) == 0)
            for (int r = 0; r < dim; r++) grad[m][r] = g[r];
    }
    double gr = 0, gT = 0, gu = 0;
    for (int d = 0; d < 3; d++) {
        gr += grad[0][d] * grad[0][d];
        gT += grad[1][d] * grad[1][d];
        for (int k = 2; k < 5; k++) gu += grad[k][d] * grad[k][d];
    }
    double m = sqrt(gr) / rho[c];
    if (sqrt(gT) / T[c] > m) m = sqrt(gT) / T[c];
    if (sqrt(gu) / sqrt(T[c]) > m) m = sqrt(gu) / sqrt(T[c]);
    return kn / rho[c] * m;
}

int orc_kn_local(const orc_problem *p, double kn, double *out)
{
    if (!p->f) return -1; /* a problem without f storage */
    int64_t nc = p->ncells;
    double *rho = (double *)malloc((size_t)nc * sizeof(double));
    double *u = (double *)malloc((size_t)nc * 3 * sizeof(double));
    double *T = (double *)malloc((size_t)nc * sizeof(double));
    double *xc = (double *)malloc((size_t)nc * 3 * sizeof(double));
    orc_moments(p, rho, u, T);
    orc_cell_centres(p, xc, NULL);
    for (int64_t c = 0; c < nc; c++) out[c] = kn_cell(p, c, kn, rho, u, T, xc);
    free(rho); free(u); free(T); free(xc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Hermite modes. */
static void hermite4(double x, double h[4])
{
    h[0] = 1.0;
    h[1] = x;
    h[2] = (x * x - 1.0) / sqrt(2.0);
    h[3] = (x * x * x - 3.0 * x) / sqrt(6.0);
}

static double mode_value(const double hx[4], const double hy[4], const double hz[4], int m)
{
    return hx[m >> 4] * hy[(m >> 2) & 3] * hz[m & 3];
}

/* the 64 coefficients of one cell's f (and its rho, u, T into mom5 unless
 * NULL) */
static void hermite_cell(const orc_problem *p, const double *fc, double *a64, double *mom5)
{
    double rho, u[3], T;
    cell_moments(p, fc, &rho, u, &T);
    double sq = sqrt(T);
    double acc[64] = {0};
    for (int64_t v = 0; v < p->nv; v++) {
        const double *x = &p->xi[3 * v];
        double hx[4], hy[4], hz[4];
        hermite4((x[0] - u[0]) / sq, hx);
        hermite4((x[1] - u[1]) / sq, hy);
        hermite4((x[2] - u[2]) / sq, hz);
        for (int m = 0; m < 64; m++) acc[m] += fc[v] * mode_value(hx, hy, hz, m);
    }
    for (int m = 0; m < 64; m++) a64[m] = acc[m] * p->dV / rho;
    if (mom5) {
        mom5[0] = rho;
        for (int d = 0; d < 3; d++) mom5[1 + d] = u[d];
        mom5[4] = T;
    }
}

int orc_hermite_project(const orc_problem *p, const double *f, double *a, double *mom)
{
    if (!f && !p->f) return -1; /* a problem without f storage */
    const double *F = f ? f : p->f;
    for (int64_t c = 0; c < p->ncells; c++) hermite_cell(p, &F[c * p->nv], &a[c * 64], mom ? &mom[c * 5] : NULL);
    return 0;
}

int orc_hermite_target(const orc_problem *p, const double *I, const double *mom, double *o)
{
    for (int64_t c = 0; c < p->ncells; c++) {
        const double *ic = &I[c * p->nv];
        double rho = mom[c * 5], T = mom[c * 5 + 4];
        const double *u = &mom[c * 5 + 1];
        double sq = sqrt(T);
        double acc[64] = {0};
        for (int64_t v = 0; v < p->nv; v++) {
            const double *x = &p->xi[3 * v];
            double hx[4], hy[4], hz[4];
            hermite4((x[0] - u[0]) / sq, hx);
            hermite4((x[1] - u[1]) / sq, hy);
            hermite4((x[2] - u[2]) / sq, hz);
            for (int m = 0; m < 64; m++) acc[m] += ic[v] * mode_value(hx, hy, hz, m);
        }
        for (int m = 0; m < 64; m++) o[c * 64 + m] = acc[m] * p->dV / (rho * rho * sq);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* MLP 64 -> 256 -> 256 -> 256 -> 64 with SiLU. */
static const int mlp_in[4] = {64, 256, 256, 256};
static const int mlp_out[4] = {256, 256, 256, 64};

static double silu(double x) { return x / (1.0 + exp(-x)); }
static double silu_grad(double x)
{
    double s = 1.0 / (1.0 + exp(-x));
    return s * (1.0 + x * (1.0 - s));
}

static const double *layer_W(const double *params, int l)
{
    size_t off = 0;
    for (int k = 0; k < l; k++) off += (size_t)mlp_in[k] * mlp_out[k] + mlp_out[k];
    return params + off;
}

/* z[l] are pre-activations of layer l (0..3), per sample */
static void mlp_sample(const double *params, const double *x, double *z[4], double *h[4], double *y)
{
    const double *in = x;
    for (int l = 0; l < 4; l++) {
        const double *W = layer_W(params, l);
        const double *b = W + (size_t)mlp_in[l] * mlp_out[l];
        for (int o = 0; o < mlp_out[l]; o++) {
            double s = b[o];
            for (int i = 0; i < mlp_in[l]; i++) s += W[(size_t)o * mlp_in[l] + i] * in[i];
            z[l][o] = s;
            h[l][o] = l < 3 ? silu(s) : s;
        }
        in = h[l];
    }
    for (int o = 0; o < 64; o++) y[o] = h[3][o];
}

int orc_mlp_forward(int64_t n, const double *params, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; s++) {
        double zb[4][256], hb[4][256];
        double *z[4] = {zb[0], zb[1], zb[2], zb[3]}, *h[4] = {hb[0], hb[1], hb[2], hb[3]};
        mlp_sample(params, &x[s * 64], z, h, &y[s * 64]);
    }
    return 0;
}

int orc_mlp_backward(int64_t n, const double *params, const double *x, const double *t,
                     double *grad, double *loss)
{
    memset(grad, 0, (size_t)ORC_MLP_NPARAM * sizeof(double));
    double L = 0.0;
    const double scale = 2.0 / ((double)n * 64.0);
    for (int64_t s = 0; s < n; s++) {
        double zb[4][256], hb[4][256], y[64];
        double *z[4] = {zb[0], zb[1], zb[2], zb[3]}, *h[4] = {hb[0], hb[1], hb[2], hb[3]};
        mlp_sample(params, &x[s * 64], z, h, y);
        double delta[256], next[256];
        for (int o = 0; o < 64; o++) {
            double r = y[o] - t[s * 64 + o];
            L += r * r;
            delta[o] = scale * r; /* dL/dz of the linear output layer */
        }
        for (int l = 3; l >= 0; l--) {
            const double *in = l ? h[l - 1] : &x[s * 64];
            size_t off = (size_t)(layer_W(params, l) - params);
            double *gW = grad + off;
            double *gb = gW + (size_t)mlp_in[l] * mlp_out[l];
            const double *W = params + off;
            for (int o = 0; o < mlp_out[l]; o++) {
                gb[o] += delta[o];
                for (int i = 0; i < mlp_in[l]; i++) gW[(size_t)o * mlp_in[l] + i] += delta[o] * in[i];
            }
            if (l == 0) break;
            for (int i = 0; i < mlp_in[l]; i++) {
                double sacc = 0.0;
                for (int o = 0; o < mlp_out[l]; o++) sacc += W[(size_t)o * mlp_in[l] + i] * delta[o];
                next[i] = sacc * silu_grad(z[l - 1][i]);
            }
            for (int i = 0; i < mlp_in[l]; i++) delta[i] = next[i];
        }
    }
    *loss = L / ((double)n * 64.0);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Learned collision with conservative projection, entropy check, fallback:
 * the application of given network outputs o, gated by the given local Kn. */
/* the learned update of one cell's f (in place): gate on its local Kn,
 * reconstruction of the network term o64 in the cell's Hermite basis,
 * conservative correction, entropy check; qhs_c (the plain hard-sphere term
 * of the cell, may be NULL) replaces the term where the gate or a check
 * rejects it.  -1 if it is rejected and there is no plain term. */
static int learned_cell(const orc_problem *p, double *f, double knl, const double *o64, double kn_threshold,
                        const double *qhs_c, double dt, double kn, int32_t *used, double *q_c)
{
    int64_t nv = p->nv;
    double rho, u[3], T;
    cell_moments(p, f, &rho, u, &T);
    double sq = sqrt(T);
    double *Q = (double *)malloc((size_t)nv * sizeof(double));
    int ok = knl < kn_threshold;
    if (ok) {
        double A[25] = {0}, rhs[5] = {0}, cc[5];
        double *M = (double *)malloc((size_t)nv * sizeof(double));
        for (int64_t v = 0; v < nv; v++) {
            const double *x = &p->xi[3 * v];
            double g[3], hx[4], hy[4], hz[4];
            for (int d = 0; d < 3; d++) g[d] = (x[d] - u[d]) / sq;
            hermite4(g[0], hx);
            hermite4(g[1], hy);
            hermite4(g[2], hz);
            double s = 0.0;
            for (int m = 0; m < 64; m++) s += o64[m] * mode_value(hx, hy, hz, m);
            M[v] = maxwellian(rho, u, T, x);
            Q[v] = rho * sq * M[v] * s;
            double ph[5] = {1.0, g[0], g[1], g[2], g[0] * g[0] + g[1] * g[1] + g[2] * g[2] - 3.0};
            for (int r = 0; r < 5; r++) {
                for (int k = 0; k < 5; k++) A[r * 5 + k] += ph[r] * ph[k] * M[v] * p->dV;
                rhs[r] += ph[r] * Q[v] * p->dV;
            }
        }
        if (orc_solve(5, A, rhs, cc)) ok = 0;
        double ent = 0.0, qabs = 0.0;
        for (int64_t v = 0; v < nv && ok; v++) {
            const double *x = &p->xi[3 * v];
            double g[3];
            for (int d = 0; d < 3; d++) g[d] = (x[d] - u[d]) / sq;
            double ph[5] = {1.0, g[0], g[1], g[2], g[0] * g[0] + g[1] * g[1] + g[2] * g[2] - 3.0};
            double corr = 0.0;
            for (int r = 0; r < 5; r++) corr += cc[r] * ph[r];
            Q[v] -= M[v] * corr;
            ent += Q[v] * log(f[v] > 0.0 ? f[v] : 1e-300) * p->dV;
            qabs += fabs(Q[v]) * p->dV;
        }
        /* entropy production sum Q ln f dV non-positive (H-theorem),
         * up to the error of its evaluation.  The bound 1e-5 sum |Q| dV
         * is set by the FP32 evaluation on the device, which sums
         * Q ln(f/M) (ln M is a collision invariant, so the exact sum is
         * the same) with about 54 terms per thread: a relative error of
         * at most 54 * 2^-24 = 3.2e-6 of sum |Q| |ln(f/M)| dV, and ln(f/M)
         * is O(1) where Q is not negligible.  A term whose exact
         * production is <= 0 is therefore kept on both sides; here in
         * FP64 the invariant part sum Q ln M cancels to the correction's
         * residual (1e-12 of its scale).  An equilibrium cell, where the
         * production is zero up to rounding, passes. */
        if (ok && !(ent <= 1e-5 * qabs)) ok = 0;
        free(M);
    }
    if (!ok) {
        if (!qhs_c) { free(Q); return -1; }
        for (int64_t v = 0; v < nv; v++) Q[v] = qhs_c[v];
    }
    if (used) *used = ok;
    for (int64_t v = 0; v < nv; v++) {
        if (q_c) q_c[v] = Q[v];
        f[v] += dt / kn * Q[v];
    }
    free(Q);
    return 0;
}

/* Learned collision with conservative projection, entropy check, fallback:
 * the application of given network outputs o, gated by the given local Kn. */
int orc_learned_apply(orc_problem *p, double dt, double kn, const double *knl, const double *o,
                      double kn_threshold, int32_t *used, double *q)
{
    if (!p->f) return -1; /* a problem without f storage */
    int64_t nc = p->ncells, nv = p->nv;
    /* the plain operator for every cell (the fallback, and the yardstick of the learned error) */
    double *qhs = NULL;
    if (p->hs_start) {
        double *f0 = (double *)malloc((size_t)(nc * nv) * sizeof(double));
        memcpy(f0, p->f, (size_t)(nc * nv) * sizeof(double));
        qhs = (double *)malloc((size_t)(nc * nv) * sizeof(double));
        if (orc_hs_collide(p, 0.0, 1.0, qhs, NULL, NULL)) { free(f0); free(qhs); return -1; }
        memcpy(p->f, f0, (size_t)(nc * nv) * sizeof(double));
        free(f0);
    }
    int err = 0;
    for (int64_t c = 0; c < nc; c++)
        if (learned_cell(p, &p->f[c * nv], knl[c], &o[c * 64], kn_threshold, qhs ? &qhs[c * nv] : NULL, dt, kn,
                         used ? &used[c] : NULL, q ? &q[c * nv] : NULL))
            err = 1;
    free(qhs);
    return err ? -1 : 0;
}

/* the 64 coefficients of the Maxwellian M(rho, u, T) sampled at the nodes,
 * in its own Hermite basis (mom5 = rho, u, T) */
static void hermite_maxwellian_cell(const orc_problem *p, const double *mom5, double *a64)
{
    const double rho = mom5[0], T = mom5[4], *u = &mom5[1];
    const double sq = sqrt(T);
    double acc[64] = {0};
    for (int64_t v = 0; v < p->nv; v++) {
        const double *x = &p->xi[3 * v];
        double hx[4], hy[4], hz[4];
        hermite4((x[0] - u[0]) / sq, hx);
        hermite4((x[1] - u[1]) / sq, hy);
        hermite4((x[2] - u[2]) / sq, hz);
        const double M = maxwellian(rho, u, T, x);
        for (int m = 0; m < 64; m++) acc[m] += M * mode_value(hx, hy, hz, m);
    }
    for (int m = 0; m < 64; m++) a64[m] = acc[m] * p->dV / rho;
}

/* The whole learned update: local Kn, projection, network, application.
 * The network term is o(a) - o(a_M), a_M the projection of the cell's own
 * Maxwellian M(rho, u, T) sampled at the nodes (in the cell's Hermite
 * basis), so that the term vanishes at equilibrium. */
int orc_learned_collide(orc_problem *p, double dt, double kn, const double *params,
                        double kn_threshold, int32_t *used, double *q)
{
    if (!p->f) return -1; /* a problem without f storage */
    int64_t nc = p->ncells;
    double *knl = (double *)malloc((size_t)nc * sizeof(double));
    double *a = (double *)malloc((size_t)nc * 128 * sizeof(double));
    double *o = (double *)malloc((size_t)nc * 128 * sizeof(double));
    double *mom = (double *)malloc((size_t)nc * 5 * sizeof(double));
    orc_kn_local(p, kn, knl);
    orc_hermite_project(p, NULL, a, mom);
    for (int64_t c = 0; c < nc; c++) hermite_maxwellian_cell(p, &mom[c * 5], &a[(nc + c) * 64]);
    orc_mlp_forward(2 * nc, params, a, o);
    for (int64_t k = 0; k < nc * 64; k++) o[k] -= o[nc * 64 + k];
    int rc = orc_learned_apply(p, dt, kn, knl, o, kn_threshold, used, q);
    free(knl); free(a); free(o); free(mom);
    return rc;
}

/* One learned step (transport, Eq. 2, then the learned update with the
 * hard-sphere fallback) of selected cells from supplied rows: the rows of
 * inputs must cover the cells' face neighbours and theirs (the local Kn
 * reads the moments of the neighbours' f*).  Per-cell arithmetic as in the
 * full step; knl_out and used (may be NULL) get the cells' local Kn and
 * gate outcome. */
int orc_step_cells_learned(const orc_problem *p, int64_t n, const int64_t *cells, int64_t ninp,
                           const int64_t *inputs, const double *fin, double dt, double kn, const double *params,
                           double kn_threshold, double *knl_out, int32_t *used, double *out)
{
    if (!p->hs_start) return -1;
    const int64_t nv = p->nv, nc = p->ncells;
    /* the cells whose f* the step reads: the cells and their face neighbours */
    const int64_t n1 = orc_step_inputs(p, n, cells, NULL);
    if (n1 < 0) return -1;
    int64_t *ring = (int64_t *)malloc((size_t)(n1 > 0 ? n1 : 1) * sizeof(int64_t));
    orc_step_inputs(p, n, cells, ring);
    row_table t = {ninp, inputs, fin};
    for (int64_t i = 0; i < n1; i++) {
        int miss = !row_sparse(p, &t, ring[i]);
        for (int64_t e = p->cf_start[ring[i]]; e < p->cf_start[ring[i] + 1] && !miss; e++) {
            const int64_t q = p->cf_list[e];
            if (q >= 0 && (!row_sparse(p, &t, p->cell_of_leaf[p->fm[q]]) || !row_sparse(p, &t, p->cell_of_leaf[p->fp[q]])))
                miss = 1;
        }
        if (miss) { free(ring); return -1; }
    }
    double *fs = (double *)malloc((size_t)(n1 * nv) * sizeof(double));
    double *rho = (double *)calloc((size_t)nc, sizeof(double));
    double *u = (double *)calloc((size_t)nc * 3, sizeof(double));
    double *T = (double *)calloc((size_t)nc, sizeof(double));
    double *xc = (double *)malloc((size_t)nc * 3 * sizeof(double));
    orc_cell_centres(p, xc, NULL);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n1; i++) {
        transport_cell(p, ring[i], row_sparse, &t, dt, &fs[i * nv]);
        cell_moments(p, &fs[i * nv], &rho[ring[i]], &u[3 * ring[i]], &T[ring[i]]);
    }
    row_table ts = {n1, ring, fs};
    double *a = (double *)malloc((size_t)(n > 0 ? n : 1) * 128 * sizeof(double));
    double *o = (double *)malloc((size_t)(n > 0 ? n : 1) * 128 * sizeof(double));
    double *knl = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n; i++) {
        double mom5[5];
        knl[i] = kn_cell(p, cells[i], kn, rho, u, T, xc);
        hermite_cell(p, row_sparse(p, &ts, cells[i]), &a[i * 64], mom5);
        hermite_maxwellian_cell(p, mom5, &a[(n + i) * 64]);
    }
    orc_mlp_forward(2 * n, params, a, o);
    for (int64_t k = 0; k < n * 64; k++) o[k] -= o[n * 64 + k];
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int64_t i = 0; i < n; i++) {
        double *row = &out[i * nv];
        memcpy(row, row_sparse(p, &ts, cells[i]), (size_t)nv * sizeof(double));
        /* the plain term of the cell: the hard-sphere update with dt = 0, Kn = 1 */
        double *f0 = (double *)malloc((size_t)nv * sizeof(double));
        double *qhs = (double *)malloc((size_t)nv * sizeof(double));
        memcpy(f0, row, (size_t)nv * sizeof(double));
        if (hs_cell(p, f0, 0.0, 1.0, qhs, NULL, NULL)) err = 1;
        else if (learned_cell(p, row, knl[i], &o[i * 64], kn_threshold, qhs, dt, kn, used ? &used[i] : NULL, NULL))
            err = 1;
        if (knl_out) knl_out[i] = knl[i];
        free(f0);
        free(qhs);
    }
    free(ring); free(fs); free(rho); free(u); free(T); free(xc); free(a); free(o); free(knl);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------------------ */
/* Mesh adaptation with f carried over.  The paper's trees are refined and
 * coarsened as the solution evolves (Sec. 2.1, Sec. 5) and the advection
 * stencils are rebuilt on every such change (Sec. 3.1, step 4).  Refinement
 * hands each new cell the distribution of the old leaf that contains it
 * (piecewise-constant injection); coarsening gives a merged parent the mean
 * of its children's distributions (equal volumes, so mass, momentum and
 * energy are kept).  Both replace the leaves, rebuild cells and faces and
 * keep the velocity grid, the freestream and the hard-sphere tables. */

static void free_mesh(orc_problem *p)
{
    free(p->lv); free(p->cell_of_leaf); free(p->leaf_of_cell);
    free(p->fm); free(p->fp); free(p->fax); free(p->farea);
    free(p->cf_start); free(p->cf_list);
    free(p->bl); free(p->bother); free(p->bax); free(p->bside); free(p->bkind); free(p->barea);
    p->lv = NULL; p->cell_of_leaf = NULL; p->leaf_of_cell = NULL;
    p->fm = NULL; p->fp = NULL; p->fax = NULL; p->farea = NULL;
    p->cf_start = NULL; p->cf_list = NULL;
    p->bl = NULL; p->bother = NULL; p->bax = NULL; p->bside = NULL; p->bkind = NULL; p->barea = NULL;
    p->nleaves = p->ncells = p->nf = p->nbf = 0;
}

/* the leaves v[n] (Morton order, solid flags set) become the problem's mesh */
static int set_mesh(orc_problem *p, leaf_t *v, int64_t n)
{
    free_mesh(p);
    p->lv = v;
    p->nleaves = n;
    p->cell_of_leaf = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    p->leaf_of_cell = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!p->cell_of_leaf || !p->leaf_of_cell) return -1;
    for (int64_t a = 0; a < n; a++) {
        if (v[a].solid) p->cell_of_leaf[a] = -1;
        else { p->cell_of_leaf[a] = p->ncells; p->leaf_of_cell[p->ncells++] = a; }
    }
    return build_faces(p);
}

int orc_refine_project(orc_problem *p, const uint8_t *flag)
{
    if (!p->f) return -1; /* a problem without f storage */
    const orc_tree_spec *s = &p->spec;
    int dim = s->dim, L = p->L;
    /* split every flagged leaf below the deepest level, then balance */
    leafvec cur = {0, 0, 0};
    for (int64_t a = 0; a < p->nleaves; a++) {
        if (flag[a] && p->lv[a].lev < L) { if (push_children(&cur, &p->lv[a], dim, L)) return -1; }
        else if (push(&cur, p->lv[a])) return -1;
    }
    if (balance_fixpoint(s, &cur)) return -1;
    for (int64_t a = 0; a < cur.n; a++) cur.v[a].solid = (uint8_t)is_solid(s, &cur.v[a]);
    /* keep the old mesh's leaves and f while the new mesh is built */
    int64_t on = p->nleaves, nv = p->nv;
    leaf_t *olv = p->lv;
    int64_t *ocell = p->cell_of_leaf;
    double *of = p->f;
    p->lv = NULL;
    p->cell_of_leaf = NULL;
    p->f = NULL;
    if (set_mesh(p, cur.v, cur.n)) { free(olv); free(ocell); free(of); return -1; }
    p->f = (double *)malloc((size_t)(p->ncells * nv) * sizeof(double));
    if (!p->f) { free(olv); free(ocell); free(of); return -1; }
    for (int64_t j = 0; j < p->ncells; j++) {
        /* the old leaf holding the new cell's anchor contains the whole cell */
        int64_t a = locate(olv, on, p->lv[p->leaf_of_cell[j]].key);
        int64_t oc = ocell[a];
        const double *src = oc >= 0 ? of + oc * nv : p->finf;
        memcpy(p->f + j * nv, src, (size_t)nv * sizeof(double));
    }
    free(olv); free(ocell); free(of);
    return 0;
}

int orc_coarsen_project(orc_problem *p, const uint8_t *flag)
{
    if (!p->f) return -1; /* a problem without f storage */
    const orc_tree_spec *s = &p->spec;
    int dim = s->dim, L = p->L, nch = 1 << dim;
    int64_t on = p->nleaves, nv = p->nv;
    const leaf_t *ol = p->lv;
    /* candidate merges: nch consecutive leaves (children of one box occupy a
     * contiguous Morton range) that are all the children of one parent at or
     * above the base level, and all flagged */
    int64_t *first = (int64_t *)malloc((size_t)on * sizeof(int64_t));
    char *on_g = (char *)malloc((size_t)on + 1);
    if (!first || !on_g) return -1;
    int64_t ng = 0;
    for (int64_t q = 0; q + nch <= on;) {
        const leaf_t *a = &ol[q];
        int ok = a->lev > s->base_level;
        for (int k = 0; k < nch && ok; k++) {
            const leaf_t *b = &ol[q + k];
            ok = flag[q + k] && b->lev == a->lev;
            for (int d = 0; d < dim && ok; d++) ok = (b->i[d] >> 1) == (a->i[d] >> 1) && (b->i[d] & 1) == ((k >> d) & 1);
        }
        if (ok) { first[ng] = q; on_g[ng++] = 1; q += nch; }
        else q++;
    }
    /* undo every merge whose parent touches a leaf two or more levels finer,
     * until none is left (undoing only adds finer leaves, so the set that
     * remains is the largest consistent one, whatever the order) */
    leafvec cur = {0, 0, 0};
    int64_t *src0 = NULL, *srcn = NULL;
    for (;;) {
        free(cur.v);
        cur.v = NULL; cur.n = cur.cap = 0;
        free(src0); free(srcn);
        src0 = (int64_t *)malloc((size_t)on * sizeof(int64_t));
        srcn = (int64_t *)malloc((size_t)on * sizeof(int64_t));
        if (!src0 || !srcn) return -1;
        int64_t g = 0;
        for (int64_t q = 0; q < on;) {
            while (g < ng && first[g] < q) g++;
            if (g < ng && first[g] == q && on_g[g]) {
                leaf_t par;
                memset(&par, 0, sizeof par);
                par.lev = ol[q].lev - 1;
                for (int d = 0; d < dim; d++) par.i[d] = ol[q].i[d] >> 1;
                set_key(&par, dim, L);
                src0[cur.n] = q; srcn[cur.n] = nch;
                if (push(&cur, par)) return -1;
                q += nch;
            } else {
                src0[cur.n] = q; srcn[cur.n] = 1;
                if (push(&cur, ol[q])) return -1;
                q++;
            }
        }
        int changed = 0;
        for (int64_t a = 0; a < cur.n; a++)
            if (srcn[a] > 1 && violates_balance(s, L, cur.v, cur.n, &cur.v[a])) {
                for (g = 0; g < ng; g++)
                    if (first[g] == src0[a]) on_g[g] = 0;
                changed = 1;
            }
        if (!changed) break;
    }
    free(first); free(on_g);
    for (int64_t a = 0; a < cur.n; a++) cur.v[a].solid = (uint8_t)is_solid(s, &cur.v[a]);
    /* f of the new cells: an unchanged cell keeps its own, a merged parent
     * takes the mean over its fluid children, or the freestream if all were
     * solid */
    leaf_t *olv = p->lv;
    int64_t *ocell = p->cell_of_leaf;
    double *of = p->f;
    p->lv = NULL;
    p->cell_of_leaf = NULL;
    p->f = NULL;
    if (set_mesh(p, cur.v, cur.n)) { free(olv); free(ocell); free(of); free(src0); free(srcn); return -1; }
    p->f = (double *)calloc((size_t)(p->ncells * nv), sizeof(double));
    if (!p->f) return -1;
    for (int64_t j = 0; j < p->ncells; j++) {
        int64_t a = p->leaf_of_cell[j];
        double *dst = p->f + j * nv;
        int64_t nf = 0;
        for (int64_t k = src0[a]; k < src0[a] + srcn[a]; k++) {
            if (ocell[k] < 0) continue;
            const double *src = of + ocell[k] * nv;
            for (int64_t v = 0; v < nv; v++) dst[v] += src[v];
            nf++;
        }
        if (nf == 0) memcpy(dst, p->finf, (size_t)nv * sizeof(double));
        else for (int64_t v = 0; v < nv; v++) dst[v] /= (double)nf;
    }
    free(olv); free(ocell); free(of); free(src0); free(srcn);
    return 0;
}
