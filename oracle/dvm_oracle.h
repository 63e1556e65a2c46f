/*
 * FP64 CPU oracle for the explicit discrete-velocity (DVM) Boltzmann step on a
 * tree-based adaptive Cartesian mesh (Zabelok, Arslanbekov, Kolobov, "Adaptive
 * Kinetic-Fluid Solvers for Heterogeneous Computing Architectures", Sec. 2.1,
 * Sec. 3, Eqs. 1-6).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never does.  It shares no code, header or table with the CUDA library.
 *
 * Everything is IEEE double.  Loops follow the paper's definitions directly:
 * no blocking, no fusion.
 */
#ifndef DVM_ORACLE_H
#define DVM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Boundary kinds for the six domain sides (x-, x+, y-, y+, z-, z+). */
enum { ORC_BC_PERIODIC = 0, ORC_BC_INFLOW = 1, ORC_BC_OUTFLOW = 2, ORC_BC_WALL = 3 };

/* Refinement predicates. */
enum { ORC_PRED_NONE = 0, ORC_PRED_BALL = 1, ORC_PRED_SHELL = 2 };

typedef struct {
    int dim;            /* 2 or 3 physical dimensions                       */
    int base_level;     /* uniform starting level                           */
    int max_level;      /* deepest level a refinement may reach             */
    int pred;           /* ORC_PRED_*                                       */
    double c[3];        /* predicate centre                                 */
    double r;           /* ball radius / sphere radius                      */
    double beta;        /* shell half-width in units of the box size        */
    int solid;          /* 1: leaves whose centre is inside the sphere are solid */
    int bc[6];          /* ORC_BC_* per side; periodic must come in pairs   */
} orc_tree_spec;

typedef struct orc_problem orc_problem;

/* Number of OpenMP threads the oracle's parallel loops use. */
int orc_threads(void);
void orc_set_threads(int n);

/* SplitMix64 output number n (0-based) of the stream seeded with `seed`. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t n);

/* ---- velocity grid (Sec. 3, Sec. 3.1 steps 1-3) ---- */
int64_t orc_vgrid_size(const int n[3]);
/* xi: [Nv][3] node values in octant-block order; k: [Nv][3] axis indices */
int orc_vgrid(const int n[3], const double lo[3], const double hi[3],
              double *xi, int32_t *k, double *dV);

/* ---- tree (Sec. 2.1) ---- */
int orc_build_tree(const orc_tree_spec *spec, int64_t cap, int64_t *n,
                   uint64_t *keys, uint8_t *levels, uint8_t *solid);

/* ---- problem object ---- */
orc_problem *orc_create(const orc_tree_spec *spec, const int n[3],
                        const double lo[3], const double hi[3]);
/* The same tree and velocity grid without f storage, for trees whose f does
 * not fit in host memory: only the geometry queries, orc_set_freestream,
 * orc_dt_cfl and the selected-cell calls below apply to it. */
orc_problem *orc_create_sparse(const orc_tree_spec *spec, const int n[3],
                               const double lo[3], const double hi[3]);
void orc_destroy(orc_problem *p);
int64_t orc_nleaves(const orc_problem *p);
int64_t orc_ncells(const orc_problem *p);
int64_t orc_nv(const orc_problem *p);
int orc_get_leaves(const orc_problem *p, uint64_t *keys, uint8_t *levels, uint8_t *solid);
int orc_cell_centres(const orc_problem *p, double *xyz /* [ncells][3] */, double *h);
int64_t orc_n_faces(const orc_problem *p);
int64_t orc_n_bfaces(const orc_problem *p);
/* interior faces: leaf indices (into the Morton leaf list), axis, area */
int orc_get_faces(const orc_problem *p, int64_t *minus, int64_t *plus,
                  uint8_t *axis, double *area);
/* boundary faces: fluid leaf, axis, side (0 = -, 1 = +), kind, other leaf
 * (-1 for a domain side), area */
int orc_get_bfaces(const orc_problem *p, int64_t *leaf, uint8_t *axis,
                   uint8_t *side, uint8_t *kind, int64_t *other, double *area);

int orc_set_freestream(orc_problem *p, double rho, const double u[3], double T);
/* f_j = sum_m w[j,m] M(rho[j,m], u[j,m,:], T[j,m]) at every node */
int orc_init_maxwellian(orc_problem *p, int nmix, const double *w,
                        const double *rho, const double *u, const double *T);
int orc_get_f(const orc_problem *p, double *f);
int orc_set_f(orc_problem *p, const double *f);
double orc_dt_cfl(const orc_problem *p, double cfl);

/* One transport sub-step (Eq. 2 in flux form): f <- f* */
int orc_transport(orc_problem *p, double dt);
/* moments of the stored f: rho, u[3], T per cell */
int orc_moments(const orc_problem *p, double *rho, double *u, double *T);
/* conserved totals sum_j V_j sum_i psi_r f ΔV, r = 0..4 */
int orc_totals(const orc_problem *p, double out[5]);
/* Conservative BGK relaxation of the stored f (forward Euler).  If q is
 * non-null it receives the collision term nu (M~ - f) per element. */
int orc_bgk(orc_problem *p, double dt, double kn, double *q);
/* Entropic BGK: target exp(a . psi), psi = (1, xi, |xi|^2), with the five
 * multipliers from Newton's method so that its discrete moments equal those
 * of f (the discrete entropic equilibrium); then the same relaxation. */
int orc_bgk_entropic(orc_problem *p, double dt, double kn, double *q);

/* Hard-sphere tables (Eqs. 3-5 with the seeded trial construction). */
int orc_hs_tables(orc_problem *p, int trials, uint64_t seed);
/* The same with the trials of each node on a 5-dimensional Korobov rank-1
 * lattice of `trials` points (multiplier orc_korobov_a(trials)), shifted per
 * node by seeded uniforms modulo 1: the partner is the node of axis indices
 * floor(u_d n_d), d < 3, and omega comes from u[3], u[4]. */
int orc_hs_tables_lattice(orc_problem *p, int trials, uint64_t seed);
int64_t orc_korobov_a(int64_t M);
/* The uniform numbers u[5] of trial k (of M) at node i, as the random
 * (lattice = 0: u[0..2]) or lattice (lattice = 1: u[0..4]) construction
 * draws them. */
void orc_trial_uniforms(int lattice, uint64_t seed, int64_t i, int64_t k, int64_t M, double *u);
int64_t orc_hs_nkept(const orc_problem *p);
/* per node i: first kept trial index, count of kept trials (CSR) */
int orc_hs_get_tables(const orc_problem *p, int64_t *start, int32_t *gam,
                      int32_t *l, int32_t *m, double *b, int64_t *discarded);
/* Conservative hard-sphere collision of the stored f (Eq. 6) with forward
 * Euler.  q (optional): collision term I per element; Bout, Cout optional. */
int orc_hs_collide(orc_problem *p, double dt, double kn, double *q,
                   double *Bout, double *Cout);

/* ---- one step of selected cells (transport, Eq. 2, then the collision
 * update), with the f rows supplied by the caller; the per-cell arithmetic is
 * that of orc_transport, orc_bgk and orc_hs_collide. ----
 * orc_step_inputs: the sorted distinct cells whose f a step of cells[0..n)
 * reads (the cells and their face neighbours); returns their count (out may
 * be NULL to size it), -1 for a cell index out of range. */
int64_t orc_step_inputs(const orc_problem *p, int64_t n, const int64_t *cells, int64_t *out);
/* out[c][v] = sum_m w[c,m] M(rho[c,m], u[c,m,:], T[c,m]) at every node, for
 * nrows rows given their mixture parameters (as orc_init_maxwellian). */
int orc_maxwellian_rows(const orc_problem *p, int64_t nrows, int nmix, const double *w, const double *rho,
                        const double *u, const double *T, double *out);
/* out[i][v]: cell cells[i] after one step (coll 1: conservative BGK; 2: hard
 * sphere, tables set) from the state whose rows fin[k] belong to inputs[k]
 * (sorted, as orc_step_inputs gives them); -1 if a row the step reads is
 * missing, a cell's moments are not admissible or its system is singular. */
int orc_step_cells(const orc_problem *p, int64_t n, const int64_t *cells, int64_t ninp, const int64_t *inputs,
                   const double *fin, double dt, int coll, double kn, double *out);

/* Full steps: transport, then collision on f* (Lie splitting).
 * coll: 0 none, 1 BGK, 2 hard sphere, 4 entropic BGK. */
int orc_step(orc_problem *p, int nsteps, double dt, int coll, double kn);

/* ---- local Knudsen number (continuum-breakdown sensor, Sec. 2.3, Sec. 3.4) ----
 * Kn_loc = (Kn / rho) max(|grad rho|/rho, |grad T|/T, |grad u|/sqrt(T)) from
 * the moments of the stored f (|grad u| the Frobenius norm); gradients are
 * weighted least-squares fits over the fluid face neighbours (exact for
 * linear fields across hanging faces). */
int orc_kn_local(const orc_problem *p, double kn, double *out);

/* ---- Hermite modes (learned collision operator) ----
 * h_0 = 1, h_1 = x, h_2 = (x^2 - 1)/sqrt(2), h_3 = (x^3 - 3x)/sqrt(6);
 * mode m = 16a + 4b + c is h_a(g_x) h_b(g_y) h_c(g_z), g = (xi - u)/sqrt(T).
 * a[c][m] = sum_i f_i H_m dV / rho with (rho, u, T) the moments of f;
 * mom[c] = (rho, u, T).  f = NULL uses the stored f. */
int orc_hermite_project(const orc_problem *p, const double *f, double *a, double *mom);
/* o[c][m] = sum_i I_i H_m dV / (rho^2 sqrt(T)) for a collision term I given
 * the cell's (rho, u, T) */
int orc_hermite_target(const orc_problem *p, const double *I, const double *mom, double *o);

/* ---- MLP 64 -> 256 -> 256 -> 256 -> 64, SiLU hidden activations ----
 * params (ORC_MLP_NPARAM doubles): W1[256][64] b1[256] W2[256][256] b2[256]
 * W3[256][256] b3[256] W4[64][256] b4[64], W[out][in].  Loss: mean over the
 * n*64 outputs of (y - t)^2. */
#define ORC_MLP_NPARAM 164672
int orc_mlp_forward(int64_t n, const double *params, const double *x, double *y);
int orc_mlp_backward(int64_t n, const double *params, const double *x, const double *t,
                     double *grad, double *loss);

/* Learned collision update of the stored f: cells with Kn_loc < threshold
 * take I = rho sqrt(T) M sum_m o_m H_m (o = MLP(a) - MLP(a_M), a_M the
 * projection of the cell's Maxwellian sampled at the nodes), made exactly
 * conservative by subtracting M (c0 + c.g + c4 (|g|^2 - 3)) with the five
 * c solving the discrete moment system; a cell whose corrected term fails
 * the entropy check sum I ln f dV <= 1e-5 sum |I| dV (non-positive within
 * the rounding of its evaluation) falls back to the hard-sphere term
 * (tables must be set).  used[c] = 1 where the learned term was applied.
 * f <- f + dt/Kn I. */
int orc_learned_collide(orc_problem *p, double dt, double kn, const double *params,
                        double kn_threshold, int32_t *used, double *q);
/* The same update from given local Kn numbers knl [ncells] and network
 * outputs o [ncells][64] (orc_learned_collide = orc_kn_local, then
 * orc_hermite_project, orc_mlp_forward and this). */
int orc_learned_apply(orc_problem *p, double dt, double kn, const double *knl, const double *o,
                      double kn_threshold, int32_t *used, double *q);
/* One learned step (transport, then the learned update with the hard-sphere
 * fallback, as orc_step with no collision followed by orc_learned_collide)
 * of cells[0..n) from supplied rows; inputs (sorted) must cover the cells'
 * face neighbours and theirs, as orc_step_inputs applied twice gives them.
 * out [n][nv]; knl_out [n] and used [n] (may be NULL) get each cell's local
 * Kn and whether the learned term was kept.  -1 on a missing row, missing
 * tables or a failed update. */
int orc_step_cells_learned(const orc_problem *p, int64_t n, const int64_t *cells, int64_t ninp,
                           const int64_t *inputs, const double *fin, double dt, double kn, const double *params,
                           double kn_threshold, double *knl_out, int32_t *used, double *out);

/* Gaussian elimination with partial pivoting on an n x n system (n <= 8);
 * A is row-major and is overwritten.  Returns 0, or -1 if singular. */
int orc_solve(int n, double *A, double *b, double *x);

/* ---- mesh adaptation with f carried over (Sec. 2.1; Sec. 3.1 step 4) ----
 * flag [nleaves] marks leaves of the current Morton leaf list.
 * orc_refine_project: every flagged leaf below max_level is split, then the
 * tree is balanced 2:1 to a fixpoint; each new fluid cell takes the f of the
 * old leaf that contains it (the freestream if that leaf was solid).
 * orc_coarsen_project: every 2^dim sibling leaves that are all flagged, with
 * their parent at or above the base level, merge into the parent, unless the
 * parent would touch a leaf two or more levels finer (such merges are undone
 * until none is left); a merged parent's f is the mean of its fluid
 * children's f (the freestream if all were solid), an unchanged cell keeps
 * its f.  Both rebuild cells and faces; 0 on success. */
int orc_refine_project(orc_problem *p, const uint8_t *flag);
int orc_coarsen_project(orc_problem *p, const uint8_t *flag);

/* Lattice Boltzmann on the tree (Sec. 4): velocity sets, equilibrium, BGK.
 * Velocities in order of increasing |c|^2, ties lexicographic in
 * (c_x, c_y, c_z) with -1 < 0 < 1; c [Q][3], w [Q]. */
enum { ORC_D2Q9 = 9, ORC_D3Q19 = 19, ORC_D3Q27 = 27 };
int orc_lattice_q(int lattice);
int orc_lattice(int lattice, double *c, double *w);
/* a problem on the tree with the lattice as its velocity set (dV = 1);
 * D2Q9 needs dim 2, the others dim 3 */
orc_problem *orc_create_lattice(const orc_tree_spec *spec, int lattice);
int orc_lbm_feq(const orc_problem *p, double rho, const double u[3], double *feq);
/* the inflow ghost: feq(rho, u) */
int orc_lbm_set_inflow(orc_problem *p, double rho, const double u[3]);
int orc_lbm_init(orc_problem *p, const double *rho, const double *u /* [ncells][3] */);
int orc_lbm_moments(const orc_problem *p, double *rho, double *u);
int orc_lbm_collide(orc_problem *p, double dt, double tau);
/* nsteps of transport (Eq. 2) then BGK with forward Euler */
int orc_lbm_step(orc_problem *p, int nsteps, double dt, double tau);

#ifdef __cplusplus
}
#endif
#endif
