/*
 * libdvm — explicit discrete-velocity (DVM) Boltzmann step on a tree-based
 * adaptive Cartesian mesh, on one GB300 (sm_103a).
 *
 * Method: Zabelok, Arslanbekov, Kolobov, "Adaptive Kinetic-Fluid Solvers for
 * Heterogeneous Computing Architectures" — the quad/octree mesh with 2:1
 * balance for direct and diagonal neighbours and Morton ordering (Sec. 2.1),
 * the non-dimensional Boltzmann equation df/dt + xi.grad f = I(f,f)/Kn
 * (Sec. 3, Eq. 1), the discrete velocity method on a uniform velocity grid
 * (Sec. 3), the finite-volume advection scheme (Sec. 3.1, Eq. 2) with the
 * velocity points grouped by the signs of their components (Sec. 3.1 steps
 * 1-4), the discrete collision integral with collision frequency B, inverse
 * integral C and the five-coefficient conservative correction (Sec. 3.2,
 * Eqs. 3-6), and the BGK relaxation form (Sec. 4).
 *
 * Conventions for every entry point:
 *   - Returns a dvm_status; DVM_OK is 0 and every failure is negative.  The
 *     message of the last failure is available from dvm_last_error().
 *   - Host arrays passed in are owned by the caller and copied before the
 *     call returns; host arrays passed out are caller-allocated with the
 *     sizes stated below.
 *   - Device memory is owned by the library (cudaMalloc, or the allocator set
 *     with dvm_set_allocator) and freed by dvm_destroy.
 *   - Calls must come in the order create -> build_tree -> set_velocity_grid
 *     -> (set_collision_tables) -> init_maxwellian/set_f -> step; a call out
 *     of order returns DVM_ESTATE.
 *   - Work is queued on the stream set by dvm_set_stream (default: the legacy
 *     default stream).  dvm_step synchronises that stream once per call to
 *     read the device status word.  No kernel traps.  The waits on
 *     asynchronous bulk copies (mbarrier waits of the hard-sphere, projection
 *     and network kernels) are bounded to about a second and report
 *     DVM_ETIMEOUT.  The step kernels' CTA-internal barriers (__syncthreads,
 *     and the named barriers between the transport and solver warps of
 *     dvm_step) carry no time bound, as no hardware barrier can; they
 *     complete because both sides of every barrier act on the same record:
 *     a CTA's cells come from a global counter into slots that alternate
 *     between two solver warps, each warp takes its slots' cells in slot
 *     order (so a parity's slots, once empty, stay empty), and the barriers
 *     of a slot are used, on both sides, exactly when that slot holds a
 *     cell.
 *   - A context is not thread-safe; use one context per host thread.
 *
 * Velocity ordering (Sec. 3.1 step 1): the Nv = nx*ny*nz nodes are stored as
 * 8 contiguous sign groups o = 4[xi_x>0] + 2[xi_y>0] + [xi_z>0]; inside a
 * group, node (mx, my, mz) (m = 0 is the node nearest zero on that axis)
 * sits at ((mx*ny/2) + my)*nz/2 + mz.  f is stored [cell][velocity], cells
 * being the non-solid leaves in Morton order.
 */
#ifndef DVM_H
#define DVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dvm_ctx dvm_ctx;

typedef enum {
    DVM_OK = 0,
    DVM_EINVAL = -1,        /* bad argument                                     */
    DVM_ENOMEM = -2,        /* device or host allocation failed                 */
    DVM_ECUDA = -3,         /* a CUDA runtime call failed                       */
    DVM_ESTATE = -4,        /* call out of order                                */
    DVM_EUNSTABLE = -5,     /* non-finite or non-positive moments, singular 5x5 system, nu*dt > 1 */
    DVM_EBOUNDS = -6,       /* a table index outside its array (checked on the host) */
    DVM_ETIMEOUT = -7,      /* a bounded device wait gave up (hard-sphere tile copies) */
    DVM_ENOTIMPL = -9       /* configuration not supported by the library         */
} dvm_status;

enum { DVM_F64 = 0, DVM_F32 = 1, DVM_BF16 = 2 };
/* Collision update applied after transport (see dvm_step):
 *   DVM_COLL_NONE          free molecular flow (transport only);
 *   DVM_COLL_BGK           BGK relaxation (Sec. 4) towards the discrete
 *                          Maxwellian times a five-coefficient correction
 *                          polynomial that restores the moments of f;
 *   DVM_COLL_HS            the hard-sphere collision integral, Eqs. 3-6;
 *   DVM_COLL_LEARNED       the learned operator (dvm_set_mlp), gated by the
 *                          local Knudsen number, falling back to Eqs. 3-6;
 *   DVM_COLL_BGK_ENTROPIC  BGK relaxation towards the discrete entropic
 *                          equilibrium exp(a . (1, xi, |xi|^2)) whose moments
 *                          on the grid equal those of f (Newton's method on a,
 *                          started from the Maxwellian; the last step's
 *                          correction is applied as the polynomial, so the
 *                          moments stay exact to the solve). */
enum { DVM_COLL_NONE = 0, DVM_COLL_BGK = 1, DVM_COLL_HS = 2, DVM_COLL_LEARNED = 3, DVM_COLL_BGK_ENTROPIC = 4 };
/* Lattice Boltzmann velocity sets (Sec. 4), named by their size. */
enum { DVM_LBM_D2Q9 = 9, DVM_LBM_D3Q19 = 19, DVM_LBM_D3Q27 = 27 };
enum { DVM_BC_PERIODIC = 0, DVM_BC_INFLOW = 1, DVM_BC_OUTFLOW = 2, DVM_BC_WALL = 3 };
enum { DVM_PRED_NONE = 0, DVM_PRED_BALL = 1, DVM_PRED_SHELL = 2 };

typedef struct {
    int precision;   /* storage of f: DVM_F64 (FP64 arithmetic throughout), DVM_F32 or
                        DVM_BF16 (FP32 transport and collision arithmetic; the moment
                        sums, the Eq. 6 correction systems and their solves in
                        FP64-class arithmetic: double-float pairs of about 48 bits
                        in the step kernel, FP64 in the hard-sphere and learned
                        corrections) */
    int collision;   /* DVM_COLL_*                                                  */
    double kn;       /* Knudsen number of Eq. 1                                     */
} dvm_config;

/* Tree specification (Sec. 2.1).  The domain is [0,1]^dim.  Starting from the
 * uniform level base_level, a box of level l < max_level is split while the
 * predicate holds:
 *   DVM_PRED_BALL:  squared distance from c to the box <= r*r;
 *   DVM_PRED_SHELL: the box meets the band r - beta*h <= |x - c| <= r + beta*h
 *                   (h = 2^-l), tested on squared distances.
 * The result is then balanced 2:1 across faces, edges and corners (periodic
 * sides wrapped).  With solid = 1 a leaf whose centre is strictly inside the
 * sphere |x - c| < r is solid: it carries no f, and its faces with fluid
 * leaves are specular walls.  bc[2d], bc[2d+1] are the kinds of the minus and
 * plus sides of axis d; periodic must come in pairs. */
typedef struct {
    int dim;          /* 2 or 3                  */
    int base_level;   /* >= 1                    */
    int max_level;    /* <= 19                   */
    int pred;         /* DVM_PRED_*              */
    double c[3];
    double r;
    double beta;
    int solid;
    int bc[6];
} dvm_tree_spec;

/* Create a context.  *out receives the handle.  Mesh calls are host work;
 * the current CUDA device is first used by dvm_set_velocity_grid, which
 * returns DVM_ECUDA when no device is available. */
int dvm_create(dvm_ctx **out, const dvm_config *cfg);

/* Release all device and host memory of the context (NULL is a no-op). */
void dvm_destroy(dvm_ctx *ctx);

/* Message of the last failure on this context ("" if none). */
const char *dvm_last_error(const dvm_ctx *ctx);

/* Queue all later work on `stream` (a cudaStream_t; NULL = default stream). */
int dvm_set_stream(dvm_ctx *ctx, void *stream);

/* Route device allocations through alloc(bytes, user) / free(ptr, user)
 * (for example a framework's caching allocator).  Must be called before
 * dvm_build_tree.  Passing NULL functions restores cudaMalloc/cudaFree. */
int dvm_set_allocator(dvm_ctx *ctx, void *(*alloc_fn)(size_t, void *),
                      void (*free_fn)(void *, void *), void *user);

/* Build the balanced tree, its Morton order, the face lists and the
 * per-cell upwind stencils (Sec. 2.1; Sec. 3.1 step 4).  Host work, once per
 * mesh.  Rebuilding discards f.  DVM_EINVAL unless 1 <= base_level <=
 * max_level <= 19, and for a tree without a fluid leaf (every leaf inside
 * the solid body): there is nothing to step. */
int dvm_build_tree(dvm_ctx *ctx, const dvm_tree_spec *spec);

/* Split every leaf i with flag[i] != 0 (indices into the Morton leaf list of
 * dvm_get_leaves, nleaves entries), rebalance, and rebuild faces and
 * stencils (Sec. 3.1: the stencil tables are redone whenever the mesh
 * changes).  f is discarded. */
int dvm_refine(dvm_ctx *ctx, const uint8_t *flag, int64_t nleaves);

/* dvm_refine with f carried over (Sec. 3.1: the mesh adapts while the
 * solution runs; the stencil tables are rebuilt).  Every new cell takes the
 * f of the old cell whose leaf contains it: a split cell's children start with
 * the parent's distribution (piecewise-constant injection), which conserves
 * mass, momentum and energy exactly.  A new fluid cell inside an old solid
 * leaf, which can appear where the wall is refined, takes the freestream
 * Maxwellian.  Needs f set (DVM_ESTATE otherwise).  Allocates new f
 * buffers; the step moments are invalidated. */
int dvm_refine_project(dvm_ctx *ctx, const uint8_t *flag, int64_t nleaves);

/* Coarsening (the inverse of dvm_refine; the paper's adaptive runs refine
 * and coarsen with the flow, Sec. 2.1).  flag[nleaves] marks leaves.  Every
 * group of 2^dim sibling leaves that are all flagged, whose parent is at or
 * above the base level, merges into its parent, unless the parent would
 * then touch a leaf two or more levels finer (2:1 balance across faces,
 * edges and corners).  Groups are undone one by one until no parent breaks
 * the balance.  The parent is solid if its centre is inside the sphere (the
 * rule of the tree build).  Like dvm_refine, the mesh alone: f is cleared. */
int dvm_coarsen(dvm_ctx *ctx, const uint8_t *flag, int64_t nleaves);

/* dvm_coarsen with f carried over: an unchanged cell keeps its f, and a
 * merged parent takes the mean of its children's f over the fluid children
 * (equal volumes, so mass, momentum and energy are kept when all children
 * are fluid), or the freestream if all were solid. */
int dvm_coarsen_project(dvm_ctx *ctx, const uint8_t *flag, int64_t nleaves);

/* Local Knudsen number of every cell (the continuum-breakdown sensor, Sec.
 * 2.3 and Sec. 3.4): Kn_loc = (Kn / rho) max(|grad rho|/rho, |grad T|/T,
 * |grad u|/sqrt(T)) (the local mean free path Kn/rho over the gradient
 * length) from the moments of the stored f, each gradient a
 * face-weighted least-squares fit over the fluid face neighbours (weights
 * area / |d|^2).  knl [ncells]. */
int dvm_kn_local(dvm_ctx *ctx, double *knl);

/* Kinetic/fluid flags from the local Knudsen number: kinetic[c] = 1 where
 * Kn_loc > threshold (the cells the Boltzmann solver keeps), else 0; the
 * number of kinetic cells in *nkinetic (may be NULL). */
int dvm_flag_kinetic(dvm_ctx *ctx, double threshold, uint8_t *kinetic, int64_t *nkinetic);

/* Sizes: leaves (including solid ones), cells (non-solid leaves), interior
 * faces, boundary faces, velocity nodes (0 before set_velocity_grid).  Any
 * pointer may be NULL. */
int dvm_get_counts(const dvm_ctx *ctx, int64_t *nleaves, int64_t *ncells,
                   int64_t *nfaces, int64_t *nbfaces, int64_t *nv);

/* Leaves in Morton order: key = bit-interleaved anchor coordinates at depth
 * max_level (bit b of x -> bit dim*b, y -> dim*b+1, z -> dim*b+2), level and
 * solid flag.  Arrays of nleaves entries. */
int dvm_get_leaves(const dvm_ctx *ctx, uint64_t *keys, uint8_t *levels, uint8_t *solid);

/* Interior faces (one per fine subface between fluid leaves, across
 * periodic sides too), sorted by (axis, key(minus), key(plus)): leaf indices,
 * axis, area = (edge of the finer leaf)^(dim-1).  Arrays of nfaces entries. */
int dvm_get_faces(const dvm_ctx *ctx, int64_t *minus, int64_t *plus, uint8_t *axis, double *area);

/* Boundary faces of fluid leaves, sorted by (kind, axis, side, key(leaf),
 * key(other)): domain sides (other = -1) and walls towards solid leaves.
 * Arrays of nbfaces entries. */
int dvm_get_bfaces(const dvm_ctx *ctx, int64_t *leaf, uint8_t *axis, uint8_t *side,
                   uint8_t *kind, int64_t *other, double *area);

/* Cell centres [ncells][3] (z = 0.5 in 2D) and edge lengths [ncells]. */
int dvm_cell_centres(const dvm_ctx *ctx, double *xyz, double *h);

/* Uniform velocity grid (Sec. 3): n[d] even, lo[d] = -hi[d] (a mirror-
 * symmetric grid, so that sign groups and specular reflection map nodes to
 * nodes).  Nodes xi_d(k) = lo_d + (k + 1/2) (hi_d - lo_d)/n_d in FP64.
 * nz/2 must be a multiple of 4 (FP32/BF16) or 2 (FP64).  Allocates f. */
int dvm_set_velocity_grid(dvm_ctx *ctx, const int n[3], const double lo[3], const double hi[3]);

/* Node values in storage order, [nv][3] FP64. */
int dvm_get_velocities(const dvm_ctx *ctx, double *xi);

/* Freestream (rho, u, T) sampled as the inflow ghost Maxwellian. */
int dvm_set_freestream(dvm_ctx *ctx, double rho, const double u[3], double T);

/* f_j = sum_m w[j][m] M(rho[j][m], u[j][m][:], T[j][m]) at every node, with
 * M = rho (2 pi T)^(-3/2) exp(-|xi - u|^2 / (2T)) evaluated in FP64 on the
 * device and rounded to the storage precision.  Arrays are per cell:
 * w, rho, T [ncells][nmix], u [ncells][nmix][3]. */
int dvm_init_maxwellian(dvm_ctx *ctx, int nmix, const double *w, const double *rho,
                        const double *u, const double *T);

/* Copy f to/from the host as FP64 [ncells][nv] (converted from/to storage). */
int dvm_get_f(dvm_ctx *ctx, double *f, int64_t count);
int dvm_set_f(dvm_ctx *ctx, const double *f, int64_t count);

/* Copy the f rows of n selected cells to the host as FP64: out[i][v] = f of
 * cell cells[i] at velocity node v (out holds n * nv doubles; cells are host
 * indices in the dvm_get_f / dvm_cell_centres order, repeats allowed).  The
 * rows are gathered and converted on the device, so only n * nv values cross
 * the host link: this inspects trees whose whole f is too large to copy.
 * Device scratch is allocated for the call and freed before it returns: the
 * row indices, and up to 2^24 values of f (rows are copied in chunks of at
 * most that many values) in the storage precision and again in FP64; the
 * call synchronises the context's stream.
 * DVM_EINVAL for an index outside [0, ncells) (nothing is copied),
 * DVM_ESTATE before f is set, DVM_ENOMEM if the scratch cannot be had. */
int dvm_get_f_rows(dvm_ctx *ctx, int64_t n, const int64_t *cells, double *out);

/* Copy f to/from host memory in the storage format (ncells*nv elements of
 * 8, 4 or 2 bytes; pinned memory gives asynchronous copies on the stream). */
int dvm_upload_f(dvm_ctx *ctx, const void *host, int64_t bytes);
int dvm_download_f(dvm_ctx *ctx, void *host, int64_t bytes);

/* Device address and size in bytes of the current f buffer (read-only view
 * for inspection; valid until the next dvm_step or rebuild). */
int dvm_f_device(const dvm_ctx *ctx, void **ptr, int64_t *bytes);

/* dt = CFL * h_min / max_i sum_{d<dim} |xi_{d,i}| over the fluid cells. */
int dvm_dt_cfl(const dvm_ctx *ctx, double cfl, double *dt);

/* Hard-sphere trial tables for Eqs. 3-5 (required for DVM_COLL_HS). */
int dvm_set_collision_tables(dvm_ctx *ctx, int trials, uint64_t seed);

/* The same tables with the trials of each node on a Korobov lattice, the
 * quasi-Monte Carlo quadrature the paper cites for the collision integral
 * (Sec. 3, Ref. [5]).  Point k of a rank-1 lattice of `trials` points in
 * [0,1)^5 has generator (1, a, a^2, a^3, a^4) mod trials, where a is the odd
 * multiplier with the largest lattice spacing.  The lattice is shifted per
 * node by seeded uniforms (SplitMix64 draws 5i .. 5i+4) modulo 1.  The
 * partner is the node with axis indices floor(u_d n_d), d < 3, and omega comes
 * from u_3, u_4 as in the random tables.  Errors as dvm_set_collision_tables. */
int dvm_set_collision_tables_lattice(dvm_ctx *ctx, int trials, uint64_t seed);

/* Copy of the hard-sphere trial tables (node-major, entry e = i*trials + k,
 * nv*trials entries each): partner gamma, post-collision nodes l and m
 * (storage indices) and weight b = c (FP32; 0 for a discarded trial, whose
 * indices then point at node i).  *discarded receives the number of
 * discarded trials. */
int dvm_get_collision_tables(const dvm_ctx *ctx, int32_t *gam, int32_t *l, int32_t *m,
                             float *b, int64_t *discarded);

/* nsteps explicit steps of size dt: transport (Eq. 2), moments of f*, then
 * the collision update on f* (Lie splitting): BGK relaxation towards the
 * conservatively corrected discrete Maxwellian or the discrete entropic
 * equilibrium, or Eqs. 3-6, with forward Euler.  Returns DVM_EUNSTABLE if any cell met a non-positive density or
 * temperature, a singular correction system or nu*dt > 1. */
int dvm_step(dvm_ctx *ctx, int nsteps, double dt);

/* Moments of the stored f per cell: rho = sum f dV, u = sum xi f dV / rho,
 * T = (sum |xi|^2 f dV / rho - |u|^2) / 3.  Host arrays rho, T [ncells],
 * u [ncells][3]. */
int dvm_moments(dvm_ctx *ctx, double *rho, double *u, double *T);

/* Moments (rho, u, T) of the post-transport state f* of the last step, as
 * used by its collision update (equal, by conservation, to those of the
 * post-collision state up to storage rounding). */
int dvm_step_moments(dvm_ctx *ctx, double *rho, double *u, double *T);

/* Conservation residual of the last collision update (Sec. 3.2, Eq. 6: the
 * correction makes the discrete collision term conserve mass, momentum and
 * energy), per cell: res [ncells][5] = sum_i psi_r(xi_i) q_i dV with
 * psi = (1, xi_x, xi_y, xi_z, |xi|^2), where q is the collision term of the
 * update f <- f* + dt q (BGK and entropic BGK: q = nu (M~ - f*)) or
 * f <- f* + dt/Kn q (hard sphere, learned: q = I), the term defined by the
 * update's per-axis tables and its correction coefficients.  The sums and the
 * 5x5 solve behind it are formed in FP64-class arithmetic (double-float or
 * FP64) on the device, so res measures how far the defined term is from
 * conserving exactly; the FP32 evaluation of q at each node and the store of
 * f round like FP32 storage and are not part of it.  Cells whose update was
 * refused (non-positive moments) hold 0.  DVM_ESTATE before the first
 * collision step, or after dvm_step_partitioned (which does not record it).
 * Synchronises the stream. */
int dvm_step_residual(dvm_ctx *ctx, double *res);

/* Phase timing of dvm_step (a diagnostic, off by default).  With enable != 0
 * every later step records CUDA events on the stream between its phases and
 * waits for the last one (one host synchronisation per step), adding the
 * phase times to three totals in ms: [0] the transport launch (for BGK and
 * entropic BGK the whole fused step), [1] the collision kernels (hard sphere:
 * the B, C and correction kernels; learned: sensor, projection, network and
 * application), [2] the hard-sphere update of the cells the learned operator
 * left over.  Enabling or disabling resets the totals. */
int dvm_set_timing(dvm_ctx *ctx, int enable);

/* The phase totals ms[3] and the number of steps behind them (steps may be
 * NULL); the totals are reset. */
int dvm_step_timing(dvm_ctx *ctx, double *ms, int64_t *steps);

/* ---- learned collision operator: the network --------------------------------
 * 64 -> 256 -> 256 -> 256 -> 64 multilayer perceptron with SiLU hidden
 * activations (not in the paper).  Parameters are a flat FP32 vector of
 * DVM_MLP_NPARAM values: W1[256][64] b1[256] W2[256][256] b2[256]
 * W3[256][256] b3[256] W4[64][256] b4[64], W[out][in].  The device keeps
 * FP32 master weights and BF16 copies; inference and training run on the
 * tensor cores with BF16 operands and FP32 accumulation.  Host arrays are
 * caller-owned; x and t are [n][64] FP32 rows. */
#define DVM_MLP_NPARAM 164672

/* Set (and reset the optimiser state of) the network's weights. */
int dvm_learned_set_weights(dvm_ctx *ctx, const float *params);

/* Copy the FP32 master weights out. */
int dvm_learned_get_weights(dvm_ctx *ctx, float *params);

/* y = MLP(x) for n rows (x rounded to BF16, BF16 activations). */
int dvm_mlp_forward(dvm_ctx *ctx, const float *x, int64_t n, float *y);

/* Mean squared error over the n*64 outputs against targets t and, if grad
 * is not NULL, its gradient with respect to the parameters. */
int dvm_mlp_loss_grad(dvm_ctx *ctx, const float *x, const float *t, int64_t n, float *grad, double *loss);

/* Train on (x, t) with Adam (beta 0.9/0.999, eps 1e-8): `epochs` passes over
 * a seeded permutation of the rows in batches of `batch` rows.  *loss
 * receives the mean training loss of the last epoch. */
int dvm_learned_train(dvm_ctx *ctx, const float *x, const float *t, int64_t n, int epochs, int batch,
                      double lr, uint64_t seed, double *loss);

/* ---- learned collision operator: the step ------------------------------------
 * DVM_COLL_LEARNED steps (FP32 storage; every n even, at most 32, n_z/2 a
 * multiple of 4; hard-sphere tables, network weights and the threshold
 * set) replace the collision update of Eqs. 3-6 by, per cell:
 *   1. the local Knudsen number Kn_loc = (Kn/rho) max(|grad rho|/rho,
 *      |grad T|/T, |grad u|/sqrt(T)) (gradients by face-weighted least
 *      squares over the face neighbours, w = A/|d|^2);
 *   2. if Kn_loc < threshold: a_m = sum_i f_i H_m(c_i) dV / rho on the 64
 *      tensor Hermite modes H_m = He_a(c_x) He_b(c_y) He_c(c_z), a, b, c < 4
 *      (orthonormal probabilists' Hermite, m = 16a + 4b + c), with
 *      c = (xi - u)/sqrt(T); o = network(a) - network(a_M), a_M the same
 *      projection of the cell's Maxwellian M(rho, u, T) sampled at the
 *      nodes (so that the term vanishes at equilibrium);
 *      Q_i = M_i (rho sqrt(T) sum_m o_m H_m(c_i) - sum_r d_r phi_r(c_i)),
 *      phi = (1, c, |c|^2 - 3), d such that Q carries no mass, momentum or
 *      energy (the correction form of Eq. 6, solved in FP64 and accepted
 *      only if its residual is below 1e-12 of the system's scale);
 *      accepted if sum_i Q_i ln f_i <= 1e-5 sum_i |Q_i| (entropy production
 *      non-positive within its rounding; f_i <= 0 read as 1e-300):
 *      f += dt/Kn Q;
 *   3. every other cell: the hard-sphere update of Eqs. 3-6.
 * The paper has no learned operator; it is the network, gating and checks
 * of this library. */

/* Knudsen threshold below which a cell may use the learned term. */
int dvm_learned_configure(dvm_ctx *ctx, double kn_threshold);

/* One learned collision update (no transport) of the stored f in place,
 * with its intermediate results: host arrays (each may be NULL) knl
 * [ncells] FP64, a and o [ncells][64] (o = network(a)), used [ncells] (1 = learned term
 * applied), q [ncells][nv] (the applied learned term; 0 in cells that fell
 * back).  o_in (host [ncells][64], may be NULL) replaces the network
 * term o(a) - o(a_M).  Moments come from the stored f in FP64. */
int dvm_learned_collide(dvm_ctx *ctx, double dt, const float *o_in, double *knl, float *a, float *o,
                        int32_t *used, float *q);

/* Training pairs from the stored f (FP32 storage, hard-sphere tables set):
 * a [ncells][64] as above and the target o [ncells][64] =
 * sum_i I_i H_m(c_i) dV / (rho^2 sqrt(T)), I the hard-sphere term of
 * Eqs. 3-6 (the inverse of the reconstruction in step 2 up to the
 * correction).  f is not changed. */
int dvm_learned_pairs(dvm_ctx *ctx, float *a, float *o);

/* Number of cells that fell back to the hard-sphere operator in the last
 * learned collision update (synchronises the stream). */
int dvm_learned_fallback_count(dvm_ctx *ctx, int64_t *n);

/* ---- Morton-range partition (Sec. 3.3) -----------------------------------
 * The multi-GPU decomposition of the step: the Morton-ordered cells split into
 * nparts contiguous ranges of equal work (every cell carries Nv velocities;
 * the first ncells % nparts ranges hold one cell more), and the upwind halo
 * of each range, the cells outside it that its advection stencils read. */

/* Range [*c0, *c1) of part `part` and its halo: *nghost cells, written to
 * ghosts (ascending global cell indices, capacity cap; may be NULL).  Host
 * work, after dvm_build_tree; no device is touched.  DVM_EINVAL for
 * nparts < 1, part outside [0, nparts), nparts > ncells or cap too small. */
int dvm_partition_info(const dvm_ctx *ctx, int nparts, int part, int64_t *c0, int64_t *c1, int64_t *nghost,
                       int64_t *ghosts, int64_t cap);

/* The same with a cost per cell (Sec. 3.3: the SFC pieces carry equal work,
 * with kinetic cells far heavier than fluid ones): weights [ncells], finite
 * and >= 0.  Range p ends before the first cell where the weight up to that
 * cell's middle passes (p + 1) W / nparts (W the total), every range holding
 * at least one cell.  Each cut then lies within half the largest single
 * weight of its target, and each range's weight within the largest single
 * weight of W / nparts, unless a range had to be cut short to leave a cell
 * for each later range.  Arguments and errors as dvm_partition_info. */
int dvm_partition_weighted(const dvm_ctx *ctx, int nparts, const double *weights, int part, int64_t *c0,
                           int64_t *c1, int64_t *nghost, int64_t *ghosts, int64_t cap);

/* nsteps steps of the stored f (transport and BGK collisions only) run as
 * nparts partitions on the current device, the way separate GPUs would run
 * them.  Each part holds its own cells, a copy of its halo and the inflow
 * ghost in buffers of its own.  Before every step the halo rows are copied
 * from their owners' buffers: this is the exchange a multi-GPU run makes
 * between ranks.  Each part then runs the step kernel on its own cells.  The
 * result (f and the step moments) is copied back into the context's state,
 * bit-identical to dvm_step.  Allocates and frees the part buffers per call
 * (about twice the f of the mesh).  Errors as dvm_step; DVM_ENOTIMPL for the
 * hard-sphere and learned collisions. */
int dvm_step_partitioned(dvm_ctx *ctx, int nparts, int nsteps, double dt);

/* ---- one rank of the Morton-range partition (Sec. 3.3) ---------------------
 * The multi-GPU form of the step.  nparts processes (one per GPU) each own a
 * contiguous range of the Morton-ordered cells (the ranges of
 * dvm_partition_info) and, before every step, take the current rows of their
 * upwind halo from the ranks that own them.  A rank's device holds only its
 * own cells, then its halo (ascending global index), then the inflow ghost:
 * inner cells first, then ghost cells, as in Sec. 3.3.  The library gives the
 * exchange plan and packs and unpacks the rows; moving the packed rows
 * between processes (NCCL send/recv or any other transport) and the two
 * global reductions (the minimum dt over ranks, the sum of the conserved
 * totals) are the caller's.  Every rank builds the tree from the same spec
 * (the build is deterministic).  Collisions: DVM_COLL_NONE, DVM_COLL_BGK,
 * DVM_COLL_BGK_ENTROPIC (DVM_ENOTIMPL otherwise).  Host arrays of cells
 * (centres, initial state, moments, f) cover the owned cells, in order. */
typedef struct dvm_rank dvm_rank;

/* Build the tree and the plan of rank `part` of nparts (host work, no device). */
int dvm_rank_create(dvm_rank **out, const dvm_config *cfg, const dvm_tree_spec *spec, int nparts, int part);
void dvm_rank_destroy(dvm_rank *r);
const char *dvm_rank_last_error(const dvm_rank *r);

/* Total cells of the tree, the owned range [c0, c1) and the halo size. */
int dvm_rank_info(const dvm_rank *r, int64_t *ncells_global, int64_t *c0, int64_t *c1, int64_t *nhalo);

/* The exchange with rank `peer`: *nsend owned cells that peer's stencils
 * read and *nrecv halo cells that peer owns, as ascending global cell
 * indices (arrays may be NULL for a count query).  The packed rows of
 * dvm_rank_pack / dvm_rank_unpack come in these orders, so the buffer one
 * rank sends to a peer is the one that peer unpacks. */
int dvm_rank_plan(const dvm_rank *r, int peer, int64_t *nsend, int64_t *send_cells, int64_t *nrecv,
                  int64_t *recv_cells);

int dvm_rank_set_stream(dvm_rank *r, void *stream);

/* As dvm_set_velocity_grid: allocates the rank's f (owned + halo + 1 rows,
 * two buffers) and its stencils on the current device. */
int dvm_rank_set_velocity_grid(dvm_rank *r, const int n[3], const double lo[3], const double hi[3]);
int dvm_rank_set_freestream(dvm_rank *r, double rho, const double u[3], double T);
int dvm_rank_cell_centres(const dvm_rank *r, double *xyz, double *h);
int dvm_rank_init_maxwellian(dvm_rank *r, int nmix, const double *w, const double *rho, const double *u,
                             const double *T);

/* Bytes of one packed row (nv values of the storage type). */
int dvm_rank_row_bytes(const dvm_rank *r, int64_t *bytes);

/* Queue on the rank's stream: pack the rows for `peer` into dev_buf (device,
 * nsend rows), or unpack the nrecv rows in dev_buf into the halo.  The halo
 * of the current f must be unpacked before each dvm_rank_step. */
int dvm_rank_pack(dvm_rank *r, int peer, void *dev_buf);
int dvm_rank_unpack(dvm_rank *r, int peer, const void *dev_buf);

/* The CFL step over the owned cells (the global step is the minimum over
 * ranks). */
int dvm_rank_dt_cfl(const dvm_rank *r, double cfl, double *dt);

/* One step of the owned cells (transport, moments, collision), reading the
 * halo rows as they stand.  Synchronises the stream; errors as dvm_step. */
int dvm_rank_step(dvm_rank *r, double dt);

int dvm_rank_moments(dvm_rank *r, double *rho, double *u, double *T);
int dvm_rank_get_f(dvm_rank *r, double *f, int64_t count);

/* Conserved totals of the owned cells: sum_j V_j (rho, rho u, rho (|u|^2 +
 * 3 T))_j, that is sum_j V_j sum_i psi_r f_ij dV with psi = (1, xi, |xi|^2). */
int dvm_rank_totals(dvm_rank *r, double *out);

/* Size in bytes of the fixed device scratch used by dvm_hs_collide_noalloc. */
#define DVM_HS_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Hard-sphere collision update f <- f + dt/Kn I(f) (the Eq. 3-6 operator of
 * dvm_step, without transport) on caller-owned device memory, allocating
 * nothing.  The paper has no counterpart: this entry point is for callers
 * that must not allocate device memory while they run, such as a framework
 * that owns all device memory through its own pool and hands plug-ins only
 * buffers it allocated, or a real-time loop whose memory is sized once at
 * start-up and may not grow afterwards.
 *   f       device pointer, FP32 [ncells][nv] in the library's velocity
 *           order, read and written in place (owned by the caller);
 *   ncells  number of cells in f; needs ncells * (8 nv + 40) bytes of
 *           scratch, at most DVM_HS_NOALLOC_SCRATCH_BYTES: larger sizes
 *           return DVM_EINVAL before any work is queued;
 *   dt      time step.
 * f must be 16-byte aligned (DVM_EINVAL otherwise): each cell's row is read
 * by one bulk copy.
 * Uses the context's velocity grid, collision tables, Kn and stream, all
 * set up beforehand (DVM_ESTATE otherwise; FP32 storage only).  Scratch is
 * a fixed array in the library's device image: every GPU that loads the
 * library holds it until the process exits, every call shares it (its
 * contents are those of the last call; nothing in it needs to start at
 * zero), and calls whose work overlaps on the GPU race on it.  The first
 * call on a device (and the first after that device's context has been
 * re-created, e.g. by cudaDeviceReset) looks up the array's device address.
 * Every call synchronises the stream once to read the status word.  On DVM_EUNSTABLE
 * (a singular correction, or dt/Kn max(P B) > 1) f already holds the
 * applied update, invalid as it may be: a caller that needs to roll back
 * keeps its own copy of f.  Non-positive density or temperature in a cell
 * also returns DVM_EUNSTABLE; that cell's f is left unchanged. */
int dvm_hs_collide_noalloc(dvm_ctx *ctx, float *f, int64_t ncells, double dt);

/* ------------------------------------------------------------------------
 * Lattice Boltzmann on the tree (Sec. 4).  The LBM module is the DVM solver
 * on a minimal velocity set, D2Q9 (2D trees), D3Q19 or D3Q27 (3D trees).
 *   - Velocities c_i have components in {-1, 0, 1}.  They are ordered by
 *     increasing |c|^2, ties lexicographic in (c_x, c_y, c_z) with -1 < 0 < 1.
 *   - Lattice weights w_i depend on |c|^2 only.  c_s^2 = 1/3.
 *   - Transport is the finite-volume upwind scheme of Eq. 2 on the tree's
 *     faces, with the tree's boundary conditions.  The inflow ghost is
 *     feq(rho_in, u_in); outflow takes the cell itself; a wall takes the
 *     cell's value at the velocity mirrored along the wall's axis.
 *   - Collision is f <- f - (dt/tau) (f - feq(rho, u)), with rho = sum f,
 *     rho u = sum c f and feq_i = w_i rho (1 + 3 c_i.u + 4.5 (c_i.u)^2 -
 *     1.5 |u|^2), applied after transport (Lie splitting).
 * f is stored in the context's precision, FP64 or FP32 (BF16:
 * DVM_ENOTIMPL), separately from the DVM f.  Host arrays of f are
 * [ncells][q] FP64.  Order: build_tree -> lbm_set_lattice -> (lbm_set_inflow)
 * -> lbm_init_equilibrium / lbm_set_f -> lbm_step.  A mesh change (build,
 * refine) keeps the lattice and clears f. */

/* Choose the velocity set (DVM_LBM_*) and allocate f (zero) and the upwind
 * codes.  DVM_EINVAL for an unknown set or one that does not match the
 * tree's dimension. */
int dvm_lbm_set_lattice(dvm_ctx *ctx, int lattice);

/* The upwind codes of the current tree (host work only; needs the tree,
 * not a device).  codes is [2 dim][ncells]: entry (2d + s, cell) describes
 * the upwind sources of the cell's side s (0 = minus) along axis d as a
 * 32-bit code:
 *   bits 0..26  source cell (the inflow ghost is cell ncells), or, with
 *               bit 30 set, the index in ovf of the side's first entry;
 *   bit 27      wall: the cell itself at the velocity mirrored along d;
 *   bits 28..29 m - 1, where the source's weight is m / (2^(dim-1) h) and a
 *               full side sums to 2^(dim-1); with bit 30 set, the number of
 *               entries - 1 (entries in ovf use the same format without
 *               bit 30);
 *   bit 30      overflow.
 * *novf receives the number of overflow entries; codes and ovf may be NULL
 * (size query). */
int dvm_lbm_get_codes(const dvm_ctx *ctx, uint32_t *codes, uint32_t *ovf, int64_t *novf);

/* A velocity set without a context: *q its size, c [q][3] and w [q] (any
 * pointer may be NULL).  DVM_EINVAL for an unknown set. */
int dvm_lbm_lattice(int lattice, int *q, int32_t *c, double *w);

/* The velocity set: c [q][3] and w [q] (q = the set's size). */
int dvm_lbm_get_velocities(const dvm_ctx *ctx, int32_t *c, double *w);

/* q, the row stride ld of the device f ([q][ld], ld >= ncells + 1) and the
 * number of overflow upwind entries (sides with 2 or 4 finer sources);
 * any pointer may be NULL. */
int dvm_lbm_info(const dvm_ctx *ctx, int *q, int64_t *ld, int64_t *noverflow);

/* Inflow ghost feq(rho, u) (default rho 1, u 0). */
int dvm_lbm_set_inflow(dvm_ctx *ctx, double rho, const double u[3]);

/* f = feq(rho[c], u[c][:]) in every cell, in FP64 rounded to storage. */
int dvm_lbm_init_equilibrium(dvm_ctx *ctx, const double *rho, const double *u);

/* Copy f to/from the host as FP64 [ncells][q]; count = ncells * q. */
int dvm_lbm_set_f(dvm_ctx *ctx, const double *f, int64_t count);
int dvm_lbm_get_f(dvm_ctx *ctx, double *f, int64_t count);

/* dt = CFL * h_min / max_i sum_{d<dim} |c_{i,d}|. */
int dvm_lbm_dt_cfl(const dvm_ctx *ctx, double cfl, double *dt);

/* nsteps steps of transport (Eq. 2) then lattice BGK, one fused kernel per
 * step.  DVM_EUNSTABLE without stepping if dt/tau > 1, and after the steps
 * if a cell met rho <= 0 or non-finite moments.  Synchronises the stream
 * once per call. */
int dvm_lbm_step(dvm_ctx *ctx, int nsteps, double dt, double tau);

/* rho [ncells] and u [ncells][3] of the stored f, in FP64. */
int dvm_lbm_moments(dvm_ctx *ctx, double *rho, double *u);

/* Number of kernel launches the library has queued in this process. */
int dvm_launch_count(int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
