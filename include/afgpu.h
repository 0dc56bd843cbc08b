/*
 * afgpu.h -- C interface of libafgpu, a GB300 (sm_103a) implementation of
 * the geometric multigrid method on quadtree/octree AMR grids of
 * Teunissen & Ebert, "Afivo" (arXiv:1701.04329).
 *
 * Problem (Sec. 3, Eq. mg-discr-equation): A_h(u_h) = rho_h on [0,1]^D, with
 * A the Laplacian or div(eps grad u) (Sec. 3.4-3.5, afg_set_operator),
 * D = 2 or 3, with Dirichlet, Neumann or periodic domain sides (without a
 * Dirichlet side: the compatible, mean-zero solution), discretised on a
 * tree of boxes of N^D cells (Sec. 1.3, 2.1).  A tree's level 1 may be a
 * block of root boxes (domain [0,r_x] x [0,r_y] (x [0,r_z])).  The library
 * holds the tree, its per-level box lists and all field data on the GPU;
 * every operator of
 * the solve (ghost cells, red-black Gauss-Seidel, residual, restriction,
 * prolongation, norms) is a CUDA kernel of this library.
 *
 * Conventions
 * -----------
 * - Every function returns an int status (AFG_OK = 0 or a negative error);
 *   afg_last_error() gives a message for the calling thread.  A call that
 *   fails on its arguments leaves the handle unchanged.
 * - Handles are opaque and not thread-safe; use one handle per host thread.
 * - Tree-building calls (create, refine, adapt, cell/face centres, export)
 *   work on HOST memory and need no GPU.
 * - Field calls take DEVICE pointers (cudaMalloc'd or torch CUDA tensors).
 *   They are enqueued on the handle's stream (afg_set_stream, default the
 *   legacy default stream) and the pointers must stay valid until that work
 *   has finished.  Calls returning host values (norms, stats) synchronise.
 * - A handle's device data lives on one CUDA device: for a tree, the device
 *   current at its first field call; for a forest, the device current at
 *   afg_forest_create.  Every later call on the handle runs on that device
 *   (the library makes it current for the call and restores the caller's
 *   device on return), so pointers and streams given to it must belong to it.
 * - Device memory of the library (tree metadata, field workspaces) comes from
 *   cudaMalloc, or from the caller's allocator (afg_set_allocator).
 * - Leaf data order ("canonical"): leaf boxes by level ascending, Morton
 *   order (x lowest bit) of the spatial index within a level; cells of a box
 *   lexicographic with x fastest.  Boundary faces: leaf boxes in the same
 *   order, sides -x,+x,-y,+y(,-z,+z), face cells lexicographic over the two
 *   tangential axes, lower axis fastest.  For a forest, tree 0's data
 *   first, then tree 1's, ...
 * - After afg_adapt all field data on the tree is invalid (set it again).
 */
#ifndef AFGPU_H
#define AFGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AFG_OK 0
#define AFG_ERR_ARG (-1)            /* invalid argument */
#define AFG_ERR_CUDA (-2)           /* a CUDA call failed (message names it) */
#define AFG_ERR_NOMEM (-3)          /* allocation failed */
#define AFG_ERR_STATE (-4)          /* call not valid in this state (e.g. no rhs set) */
#define AFG_ERR_NOT_CONVERGED (-5)  /* max_cycles reached above rel_tol (results are valid) */
#define AFG_ERR_TIMEOUT (-6)        /* a bounded device-side wait gave up */

#define AFG_FP64 0   /* all multigrid arithmetic in double precision (some neighbour sums are formed
                        exactly in 64-bit fixed point and rounded once: never less accurate) */
#define AFG_MIXED 1  /* FP64 residual + update around FP32 multigrid (defect correction) */

typedef struct afg_tree afg_tree;
typedef struct afg_forest afg_forest;

typedef struct {
    int n_down;        /* smoothing steps before restriction (Sec. 3.2, default 2) */
    int n_up;          /* smoothing steps after correction (default 2) */
    int n_base;        /* relaxation steps on the coarsest grid (default 4) */
    int max_cycles;    /* cycle limit for afg_solve / adjoint iterations (default 50) */
    double rel_tol;    /* stop when max|rho - A u| / max|rho| <= rel_tol (default 1e-10) */
    int precision;     /* AFG_FP64 or AFG_MIXED */
    int inner_vcycles; /* AFG_MIXED: FP32 V-cycles per outer FP64 step after the first (FMG) step,
                          1..16; 0 (default): for one tree, 2 on the first such step, then
                          chosen per step from the reduction per V-cycle measured on the step
                          before so that the step reaches rel_tol, at most a factor 1e-5 per
                          step (the FP32 solve's resolution); for forests, 2 */
    int use_graph;     /* 1: replay the cycle as a CUDA graph (default 1) */
    int threads_per_box; /* FP32 half-sweep (the mixed-precision solves): threads per box, 0 (default) or
                            one per 16-byte vector of a box's colour half, min(N^D/8, 256), or half as
                            many (two vectors per thread, twice the boxes per CTA); other values:
                            AFG_ERR_ARG.  The FP64 kernels take one thread per vector. */
} afg_mg_opts;

typedef struct {
    int cycles;            /* cycles done (FMG counts as one) */
    double rel_residual;   /* last max|r| / max|rho| */
    double max_residual;   /* last max|r| */
    double max_rho;        /* max|rho| over leaves */
    double seconds;        /* wall time of the call (device-synchronised) */
    double history[64];    /* rel_residual after each cycle, first 64 */
} afg_stats;

typedef struct {
    int dim, box_n, max_level;
    int highest_level;      /* finest level present */
    int n_boxes, n_leaves;  /* tree boxes (levels >= 1) */
    long long n_leaf_cells; /* unknowns */
    long long n_bfaces;     /* leaf faces on the domain boundary */
    int boxes_per_level[32];
    int leaves_per_level[32];
} afg_tree_info;

/* Defaults of Sec. 3.2 / 4.1: N_down = N_up = 2, N_base = 4. */
void afg_default_opts(afg_mg_opts *opts);

const char *afg_last_error(void);

/* Device memory allocator for every buffer the library allocates from now on
 * (the paper's code allocates per box on the host; this is the GPU
 * counterpart: a framework such as PyTorch passes its caching allocator so
 * that the solver's workspaces come out of its pool).  alloc(bytes, ctx)
 * returns device memory of the current device, 256-byte aligned, or NULL
 * (the library call then fails with AFG_ERR_NOMEM); dealloc(ptr, ctx) takes
 * back a pointer alloc returned, with the same device current.  A buffer is
 * always returned to the allocator that made it, also after a later
 * afg_set_allocator; before calling dealloc the library waits for the device
 * to finish its queued work (as cudaFree does), so the memory may be reused
 * at once.  Both NULL: back to cudaMalloc/cudaFree.  One of them NULL:
 * AFG_ERR_ARG.  Process-wide and not synchronised with other threads: set it
 * before creating handles.  Pinned host buffers (a few bytes per handle for
 * norms read back) still come from cudaMallocHost. */
int afg_set_allocator(void *(*alloc)(size_t bytes, void *ctx), void (*dealloc)(void *ptr, void *ctx), void *ctx);

/* ---- tree (Sec. 2.1-2.3) ------------------------------------------------ */

/* Create a tree on [0,1]^dim with one root box of box_n^dim cells (level 1).
 * dim in {2,3}; box_n in {4,8,16}; 1 <= max_level <= 21 (3D) or 30 (2D). */
int afg_tree_create(int dim, int box_n, int max_level, afg_tree **out);

/* Create a tree whose level 1 is a block of root boxes (Sec. 2.2: the coarse
 * grid of a non-square domain holds several boxes): nroot (host memory, dim
 * ints, each in [1, 64]) root boxes per axis, each the unit square/cube, so
 * the domain is [0,nroot[0]] x [0,nroot[1]] (x [0,nroot[2]]).  Root boxes
 * come first in the canonical box order (Morton order of their indices).
 * Every call accepts such trees: below level 1 the coarse grids of N/2, ...,
 * 2 cells hold one box per root, connected like the roots (Sec. 3.2: the
 * coarsest grid holds several boxes, relaxed together).  A single tree whose
 * block fits one CTA's shared memory (227 KB on GB300: per grid of M = 2, 4,
 * ..., N cells per root, 4 FP64 arrays of (r_x M + 2)(r_y M + 2)
 * (x (r_z M + 2)) values plus the face data of the non-periodic sides -- up
 * to 8 x 8 roots of 8^2 boxes, 4 x 4 of 16^2, 6 x 1 x 1 or 3 x 2 x 1 of 8^3,
 * no block of 16^3 boxes) solves them in that CTA, one launch per cycle;
 * larger blocks, every tree of a forest that holds a block tree, and a tree
 * given a variable-coefficient operator or another prolongation before its
 * data (afg_set_operator, afg_set_prolongation; afterwards AFG_ERR_STATE
 * where the block solve was chosen) run them as device boxes through the
 * per-level kernels, like the finer levels.  Singular problems take trees
 * of one root box.  AFG_ERR_ARG when nroot[a] << (max_level-1) exceeds
 * 2^21. */
int afg_tree_create_roots(int dim, int box_n, int max_level, const int *nroot, afg_tree **out);
int afg_tree_destroy(afg_tree *t);

/* CUDA stream (cudaStream_t) for all device work of this tree; NULL = default. */
int afg_set_stream(afg_tree *t, void *cuda_stream);

/* Refine every leaf until all leaves are at least on `level` (Sec. 1.3). */
int afg_refine_uniform(afg_tree *t, int level);

/* Leaf cell centres, canonical order, dim doubles per cell (host memory). */
int afg_cell_centers(const afg_tree *t, double *xyz_host);

/* The same leaf cell centres written into device memory (dim doubles per
 * leaf cell, n_leaf_cells * dim in all) by a kernel on the tree's stream. */
int afg_cell_centers_device(afg_tree *t, double *xyz_dev);

/* Centres of the leaf boundary faces, canonical face order (host memory). */
int afg_face_centers(const afg_tree *t, double *xyz_host);

/* Level of every leaf box, canonical order (host memory). */
int afg_leaf_levels(const afg_tree *t, int32_t *levels_host);

/* Mesh adaptation (Sec. 2.3).  flags: one int8 per leaf cell in canonical
 * order, +1 refine, 0 keep, -1 derefine (host memory).  Rules: a box with a
 * flagged cell is refined (not beyond max_level); same-level leaves,
 * diagonal ones included, within n_buf cells of such a cell are refined too;
 * coarser neighbours of a refined box are refined for 2:1 balance (faces,
 * edges and corners); the 2^D children of a box are removed when all their
 * cells are flagged -1, none of them is refined, and no same-level
 * neighbour of the box has a child that is or becomes refined.  The level
 * changes by at most one per call.  0 <= n_buf <= box_n. */
int afg_adapt(afg_tree *t, const int8_t *flags_host, int n_buf, int *n_added, int *n_removed);

/* Mesh adaptation that carries the solution along (Sec. 2.3: prolongation
 * and restriction are applied when the mesh changes): the tree is adapted as
 * by afg_adapt, and the current solution on the device moves to the new
 * leaves -- a leaf that stays keeps its values, a box whose children are
 * removed gets their mean (Sec. 2.5), and the children of a refined leaf are
 * prolonged from it with `scheme` (AFG_PROLONG_*), its ghost values filled
 * as in the solver (the stored boundary data, the refinement-boundary scheme
 * of Sec. 3.3, and for the bi/trilinear scheme the edge/corner ghosts of
 * Sec. 2.4).  The other field data (rho, boundary data, eps) must be set
 * again.  Needs the tree's field data on the device (AFG_ERR_STATE
 * otherwise); synchronises the tree's stream. */
int afg_adapt_transfer(afg_tree *t, const int8_t *flags_host, int n_buf, int scheme, int *n_added, int *n_removed);

/* Refinement flags computed on the device (the criterion of Sec. 4.1 is of
 * this form: refine where h^2 |rho| exceeds a threshold): for every leaf
 * cell, with h its cell size, flags = +1 where |f| h^power > tau_refine,
 * -1 where |f| h^power < tau_coarsen, 0 elsewhere.  f_dev: a leaf field
 * (n_leaf_cells doubles, canonical order), flags_dev: n_leaf_cells int8,
 * both device memory, on the tree's stream; copy the flags to the host for
 * afg_adapt / afg_adapt_transfer.  AFG_ERR_ARG unless 0 <= power <= 8 and
 * tau_coarsen <= tau_refine. */
int afg_flag_cells(afg_tree *t, const double *f_dev, int power, double tau_refine, double tau_coarsen,
                   int8_t *flags_dev);

int afg_info(const afg_tree *t, afg_tree_info *out);

/* Tree arrays in canonical box order (host memory): level[n], spatial index
 * idx[n*dim] (1-based, Sec. 2.1), parent[n], children[n*2^dim] (child c has
 * offset bit a = (c>>a)&1), neighbours[n*(3^dim-1)] in lexicographic
 * (dz,dy,dx) order with x fastest, centre skipped.  -1 = no box, -2 =
 * physical boundary.  Any pointer may be NULL. */
int afg_export_tree(const afg_tree *t, int32_t *level, int32_t *idx, int32_t *parent,
                    int32_t *children, int32_t *neighbours);

/* Boundary type of each domain side, types[2*dim] in the order -x,+x,-y,+y
 * (,-z,+z): AFG_BC_DIRICHLET, AFG_BC_NEUMANN or AFG_BC_PERIODIC (Sec. 2 and
 * Sec. 3 allow Dirichlet, Neumann, periodic or a mix, through ghost cells).
 * On a Neumann side the boundary datum (afg_set_dirichlet) is the outward
 * normal derivative at the face centre and the ghost is u + h b; on a
 * Dirichlet side it is the value and the ghost 2 b - u.  Periodic applies to
 * both sides of an axis and is a property of the connectivity (Sec. 2.2: the
 * box beyond the last one is the first): those sides carry no boundary faces,
 * and periodicity can only be switched while the tree is its root boxes alone
 * (set it before refining).  Without a Dirichlet side the problem is
 * singular (constants are the null space): the solver then solves
 * A u = rho - c, c = (sum h^D rho - sum over Neumann leaf faces h^(D-1) b) /
 * sum h^D, which makes the source compatible (Sec. 4.4's gravity problem
 * subtracts the mean source), and returns the solution of zero
 * volume-weighted mean (in a forest each such tree on its own: its c and its
 * mean from its own leaves); such trees take one root box and the
 * Laplacian, and have no adjoint.  AFG_ERR_ARG for any violation, with the
 * tree unchanged.  Host call; a change discards the device fields, so set rho and
 * the boundary data after it.  Default: all sides Dirichlet.  Trees of a
 * forest keep the types they had when the forest was created. */
#define AFG_BC_DIRICHLET 0
#define AFG_BC_NEUMANN 1
#define AFG_BC_PERIODIC 2
int afg_set_boundary_types(afg_tree *t, const int *types_host);

/* ---- fields (device memory, enqueued on the tree's stream) ------------- */

/* Source term rho on leaf cells (n_leaf_cells doubles). */
int afg_set_rhs(afg_tree *t, const double *rho_leaf_dev);
/* Boundary data at the leaf boundary face centres (n_bfaces doubles):
 * Dirichlet values (ghost 2 b - u, Sec. 2.4) or, on Neumann sides, outward
 * normal derivatives (ghost u + h b).  Coarse boxes use face averages.
 * Without this call the boundary data is zero. */
int afg_set_dirichlet(afg_tree *t, const double *b_face_dev);
/* Operator of the tree (Sec. 3.4-3.5).  AFG_OP_LAPLACE (default): the
 * Laplacian.  AFG_OP_VAR: div(eps grad u) with eps > 0 per leaf cell; the
 * flux through a face between cells of coefficients e1 and e2 is the
 * harmonic mean 2 e1 e2 / (e1 + e2) times the difference quotient (Sec. 3.4).
 * AFG_OP_VAR_RZ (2D only): the same in cylindrical (r,z) coordinates with
 * r = x, (1/r) d/dr (r eps du/dr) + d/dz (eps du/dz): the r-faces are weighted
 * by r_face / r_cell, so the -x side (the axis r = 0) carries no flux (Sec.
 * 3.5).  Coarse cells take the mean of their children's eps; in (r,z) every
 * restriction (u, residual, eps) is the mean weighted by the children's r.
 * Ghost eps: the same-level neighbour's, the coarse cell's across a
 * refinement boundary, the cell's own at the domain boundary; Neumann data
 * stays the normal derivative of u (flux eps b).  The coarse-grid correction
 * keeps the linear prolongation.  Host call; changing it keeps the field data
 * but requires afg_set_eps again.  AFG_ERR_ARG for an unknown op, (r,z) on a
 * 3D tree or with a periodic -x side; AFG_ERR_STATE on a tree of several
 * root boxes whose data were set for the one-CTA block solve (set the
 * operator first).  Not covered with these operators: afg_adjoint and
 * afg_forest_residual_norms_noalloc (AFG_ERR_STATE), afg_time_kernel. */
#define AFG_OP_LAPLACE 0
#define AFG_OP_VAR 1
#define AFG_OP_VAR_RZ 2
int afg_set_operator(afg_tree *t, int op);
/* Prolongation of the coarse-grid correction (Sec. 2.5): AFG_PROLONG_LINEAR
 * (default; the 2-1-1 / 1-1-1-1 scheme, exact for linear fields, the one
 * Sec. 4.1 calls first order), AFG_PROLONG_MULTILINEAR (bilinear / trilinear:
 * per axis weight 3/4 for the nearer coarse cell, 1/4 for the farther one;
 * it reads the coarse difference's edge and corner ghosts, Sec. 2.4: copied
 * from the diagonal same-level neighbour, else extrapolated linearly) or
 * AFG_PROLONG_ZEROTH (the coarse cell's value).  With a non-default scheme
 * every level, the coarse grids below the root included, runs on the
 * per-level kernels.  Host call; AFG_ERR_ARG for an unknown scheme;
 * AFG_ERR_STATE on a tree of several root boxes whose data were set for the
 * one-CTA block solve (set the scheme first). */
#define AFG_PROLONG_LINEAR 0
#define AFG_PROLONG_MULTILINEAR 1
#define AFG_PROLONG_ZEROTH 2
int afg_set_prolongation(afg_tree *t, int scheme);

/* eps > 0 on leaf cells (n_leaf_cells doubles, canonical order, device
 * memory): stored on the leaves and restricted to every coarser level. */
int afg_set_eps(afg_tree *t, const double *eps_leaf_dev);

/* Initial guess / warm start on leaf cells; without it the guess is zero. */
int afg_set_solution(afg_tree *t, const double *u_leaf_dev);
int afg_get_solution(const afg_tree *t, double *u_leaf_dev);

/* ---- multigrid (Sec. 3) -------------------------------------------------- */

/* One FMG cycle (Sec. 3.2) from the current solution. */
int afg_fmg(afg_tree *t, const afg_mg_opts *opts, afg_stats *stats);
/* One FAS V-cycle (Sec. 3.2) from the finest level. */
int afg_vcycle(afg_tree *t, const afg_mg_opts *opts, afg_stats *stats);
/* FMG, then V-cycles until rel_tol (or max_cycles: AFG_ERR_NOT_CONVERGED).
 * opts->precision selects the plain FP64 method or the mixed-precision
 * defect correction (FP64 residual and update, FP32 multigrid). */
int afg_solve(afg_tree *t, const afg_mg_opts *opts, afg_stats *stats);
/* max over leaves of |rho - A u| (composite operator) and of |rho|. */
int afg_residual_norm(afg_tree *t, double *max_abs_r, double *max_abs_rho);

/* Adjoint of the solve: given g = dL/du on leaf cells, solve K^T lambda = g
 * for the transposed composite operator (FP64) and return lambda = dL/drho
 * (leaf cells) and dL/db = -(2/h^2) lambda (Dirichlet side) or -(1/h) lambda
 * (Neumann side) at the boundary-adjacent cell of every leaf boundary face.
 * BiCGStab with the preconditioner W M W^-1 (M one V-cycle, W the cell
 * volumes); opts->precision AFG_MIXED runs M in FP32 (K^T, the recurrences
 * and the tolerance stay FP64).  Output pointers may be NULL. */
int afg_adjoint(afg_tree *t, const double *g_leaf_dev, double *lambda_leaf_dev,
                double *dL_db_face_dev, const afg_mg_opts *opts, afg_stats *stats);

/* ---- batched forest ------------------------------------------------------- */

/* A forest solves n independent trees together: per-level box lists are
 * concatenated over the trees and every kernel launch covers all of them.
 * The trees must share dim and box_n; they are copied (later changes to a
 * tree do not affect the forest).  Field data is given per forest in
 * canonical order, tree after tree. */
int afg_forest_create(int n, afg_tree *const *trees, afg_forest **out);
int afg_forest_destroy(afg_forest *f);
int afg_forest_set_stream(afg_forest *f, void *cuda_stream);
int afg_forest_counts(const afg_forest *f, long long *leaf_cells_per_tree, long long *bfaces_per_tree);
int afg_forest_set_rhs(afg_forest *f, const double *rho_dev);
int afg_forest_set_dirichlet(afg_forest *f, const double *b_dev);
/* eps of every tree (the trees' shared operator, afg_set_operator before
 * afg_forest_create), forest canonical order. */
int afg_forest_set_eps(afg_forest *f, const double *eps_dev);
int afg_forest_get_solution(const afg_forest *f, double *u_dev);
/* Solve every tree to opts->rel_tol; a converged tree is masked out of
 * later cycles.  per_tree (may be NULL) receives n stats records. */
int afg_forest_solve(afg_forest *f, const afg_mg_opts *opts, afg_stats *per_tree);

/* Autotuner for batched forests (an addition to the paper's method, whose
 * runs fix the box size and N_down = N_up = 2).  candidates[n]: forests of
 * the same problems built with different box sizes (8^2 and 16^2 cells, the
 * finest spacing equal), each with its source term and boundary data set.
 * json_in (may be NULL): {"sweeps": [[n_down, n_up], ...],
 * "vectors_per_thread": [1, 2], "reps": R}, default sweeps [[1,1],[2,2],
 * [3,3]], vectors per thread [1] (1: the FP32 half-sweep's one thread per
 * 16-byte vector of a box's colour half, 2: half as many threads per box;
 * afg_mg_opts.threads_per_box) and R = 3.  For every candidate, pair and
 * threads-per-box choice it runs afg_forest_solve with `base` (NULL: mixed
 * precision to 1e-8) -- one warm-up solve, which also captures the CUDA
 * graphs, then the fastest of R solves timed with CUDA events on the
 * forest's stream -- and writes to json_out (cap bytes, NUL-terminated) the
 * report {"objective": "unknowns_per_s", "best": ROW, "table": [ROW, ...]},
 * ROW = {"candidate", "box_n", "n_down", "n_up", "threads_per_box", "ms",
 * "unknowns", "unknowns_per_s", "converged", "worst_rel_residual",
 * "max_cycles"}.  The best row is the converged one with the most unknowns
 * per second: time to the tolerance per unknown, which compares the box
 * sizes' different meshes per unknown.  AFG_ERR_ARG on a malformed json_in
 * or a too small json_out (the message gives the size needed).  Each
 * forest's solution is overwritten. */
int afg_autotune(afg_forest *const *candidates, int n, const afg_mg_opts *base, const char *json_in,
                 char *json_out, size_t cap);

/* Allocation-free residual norms of a forest.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * where they check convergence -- e.g. a host framework that has handed the
 * whole device memory pool to its own caching allocator, or a latency-bound
 * loop in which the implicit device synchronisation of cudaMalloc/cudaFree is
 * not acceptable.  It computes the same per-tree values as the norms that
 * afg_forest_solve reports (max over leaf cells of |rho - A u| and of |rho|,
 * composite operator, for the forest's current solution) and writes them to
 * the host arrays max_abs_r[n] and max_abs_rho[n] (n = trees).  It calls no
 * cudaMalloc/cudaFree: besides the forest's own data it uses one file-scope
 * device array of 2 x 1024 eight-byte slots (16 KB held by every GPU that
 * loads the library until the process exits); forests of more than 1024
 * trees are rejected with AFG_ERR_ARG.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) and must come before
 * any stream capture.  All calls share the array and it keeps the last
 * call's contents (the slots are cleared at the start of every call), so
 * calls whose GPU work overlaps race with each other.  The forest must have
 * been created (its device data exists); the call synchronises the forest's
 * stream. */
int afg_forest_residual_norms_noalloc(afg_forest *f, double *max_abs_r, double *max_abs_rho);

/* ---- diagnostics ----------------------------------------------------------- */

/* Total number of this library's kernels launched so far in this process,
 * kernels replayed inside CUDA graphs included. */
int afg_kernel_launches(unsigned long long *count);

/* Times one kernel of the solve on its own, with CUDA events on the tree's
 * stream: `reps` launches on every box of `level` (after one warm-up launch),
 * in FP64 (fp64 = 1) or FP32.  kernel: 0 = red-black half-sweep (Sec. 3.1,
 * colours alternating; the FP32 one with homogeneous boundary data, as the
 * mixed-precision solve runs it), 1 = fused residual + restriction (level >= 2),
 * 2 = prolongation + correction (level >= 2), 3 = leaf residual with its
 * max-norm reduction (all leaves; `level` ignored), 4 = FP64 FMA issue-rate
 * probe (independent FMA chains; `level` ignored; flops count an FMA as 2;
 * the denominator of the FP64 roofline).  Returns the mean time
 * per launch, the cells covered (`cells`) and the algorithmic bytes and
 * flops of one launch.  With s = 8 (FP64) or 4 (FP32) bytes per value, per
 * cell covered: half-sweep 3s/2 bytes (other colour of u, own colour of rho
 * and u written) and (2D+1)/2 flops in FP64 (2D-1 additions and one FMA with
 * the pre-scaled source per update) or (2D+2)/2 in FP32 (and a
 * multiplication); residual + restriction 2s + 3s/2^D
 * bytes and 2D+5 flops; correction 2s + 2s/2^D bytes and 5 flops; leaf
 * residual 2s + 4 bytes (the FP32 copy of r) and 2D+3 flops.  Field contents
 * are overwritten.  Needs afg_set_rhs first. */
int afg_time_kernel(afg_tree *t, int kernel, int level, int fp64, int reps, double *avg_ms, double *bytes,
                    double *flops, long long *cells);
/* The same timing on a forest: the launches cover the level's boxes of all
 * its trees (the concatenated box list of that level). */
int afg_forest_time_kernel(afg_forest *f, int kernel, int level, int fp64, int reps, double *avg_ms, double *bytes,
                           double *flops, long long *cells);

#ifdef __cplusplus
}
#endif
#endif
