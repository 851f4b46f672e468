/*
 * mg.h -- C ABI of the GB300 quasi-matrix-free hybrid multigrid library (libmg.so).
 *
 * Implements the hot path of Weinzierl & Weinzierl, "Quasi-matrix-free hybrid
 * multigrid on dynamically adaptive Cartesian grids" (arXiv:1607.00648): in-situ
 * application of d-linear FEM stencils (9 points in 2D, 27 in 3D) in the damped
 * Jacobi smoother, the residual, BoxMG prolongation / restriction and the
 * Galerkin coarse-operator computation, every stored operator rebuilt on the fly
 * as the rediscretised stencil plus a stored hierarchical delta (Sect. 5).
 *
 * Problem (eq. "pde" with v = 0):  -div(eps grad u) = f on (0,1)^d, u = 0 on the
 * boundary, d in {2,3}, discretised on a k = 3 spacetree (Sect. 3).
 *
 * Conventions shared by every call
 * --------------------------------
 * Level layout.  Level l of the spacetree is stored as bricks: the level-l
 *   descendants of one level-(l-m) cell, m = min(l,3) in 2D and min(l,2) in 3D,
 *   so a brick has B = 3^m cells per axis.  Bricks follow the Peano curve of
 *   their root cells (Sect. 3 / App. A: depth-first order = Peano curve);
 *   inside a brick, vertex slots are lexicographic (x fastest) and padded to
 *   slots_per_brick = roundup(B^d, 32).  Slot k of brick b holds the vertex at
 *   brick_origin + lex(k).  A cell uses the slot of its lower-left vertex.
 * Vectors.  A level vector (u, b, r, eps) is a device array of n_slots entries
 *   in that order.  Only degree-of-freedom slots (EXISTS, not BOUNDARY, not
 *   HANGING) carry unknowns; every call writes 0 to the other slots of its
 *   outputs and requires 0 in the boundary slots of its inputs.
 * Ownership.  The caller owns every pointer it passes (device pointers unless
 *   the name says host); the library owns grid / hierarchy handles and all
 *   internal device storage, released by the destroy calls (which accept NULL).
 * Streams.  All device work is enqueued on the given cudaStream_t (passed as
 *   void*, NULL = legacy default stream).  Only calls that return host values
 *   (norm2_host, mg_solve) synchronise that stream.
 * Errors.  Every call returns mg_status; no C++ exception crosses the ABI.  On
 *   failure outputs are unspecified, handles stay valid, and mg_last_error()
 *   returns a thread-local message.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mg_status {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,
  MG_ERR_OOM = 2,
  MG_ERR_CUDA = 3,
  MG_ERR_NOT_CONVERGED = 4,
  MG_ERR_DIVERGED = 5,
  MG_ERR_NONFINITE = 6,
  MG_ERR_INDEFINITE_COARSE = 7,
  MG_ERR_TIMEOUT = 8,
  MG_ERR_BUDGET = 9,
  MG_ERR_UNSUPPORTED = 10
} mg_status;

/* Vertex flags (Sect. 3): a vertex is hanging if it has fewer than 2^d adjacent
 * cells on its level, refined if all its adjacent cells are refined, else
 * unrefined.  Boundary vertices carry the Dirichlet value 0. */
#define MG_V_EXISTS 1u
#define MG_V_BOUNDARY 2u
#define MG_V_HANGING 4u
#define MG_V_REFINED 8u
/* Cell flags. */
#define MG_C_EXISTS 1u
#define MG_C_REFINED 2u

typedef struct mg_grid mg_grid;
typedef struct mg_hier mg_hier;

typedef struct mg_level_info {
  int32_t level;
  int32_t dim;
  int32_t brick_edge;      /* B, cells (= owned vertices) per brick axis */
  int32_t slots_per_brick; /* roundup(B^d, 32) */
  int64_t n_bricks;
  int64_t n_slots;         /* n_bricks * slots_per_brick */
  int64_t n_dofs;          /* EXISTS && !BOUNDARY && !HANGING */
  int64_t n_cells;         /* existing cells of the level */
  int64_t n_hanging;
  int64_t slot_offset;     /* offset of this level in level-concatenated cell arrays */
  double h;                /* mesh width 3^-level */
} mg_level_info;

/* ---------------------------------------------------------------- A1 grid */

/* Build a k = 3 spacetree and flatten it into level arrays (Sect. 3, App. A).
 * dim in {2,3}; 1 <= max_level <= 8 (2D) or 6 (3D).
 * refine_masks: host array of max_level pointers (or NULL).  refine_masks[l]
 *   (or NULL = refine every existing cell) is a byte mask over the complete
 *   level l, lexicographic with x fastest, (3^l)^d entries; an existing level-l
 *   cell is refined iff its byte is non-zero.  Host memory, read during the call.
 * out: receives the grid handle (host object; destroy with mg_destroy_grid).
 * Errors: MG_ERR_INVALID_ARG for bad dim / level / NULL out, MG_ERR_OOM. */
mg_status mg_create_grid(int dim, int max_level, const uint8_t* const* refine_masks, mg_grid** out);

/* Sizes of one level (0 <= level <= max_level).  info: host struct. */
mg_status mg_grid_info(const mg_grid* grid, int level, mg_level_info* info);

/* Host copies of the level tables (each pointer nullable; host memory, sizes in
 * units of the element type):
 *  coords        n_slots*d     global integer vertex coordinates (-1 on padding slots)
 *  vflags        n_slots       MG_V_* bits
 *  cflags        n_slots       MG_C_* bits of the cell owning the slot
 *  nbr           n_slots*3^d   slot of vertex x+o, o in {-1,0,1}^d lexicographic (x
 *                              fastest), -1 outside the domain or without a slot
 *  cell_vertices n_slots*2^d   slots of the 2^d corners x+e, e in {0,1}^d lex, -1 if none
 *  hang_idx      n_slots*2^d   HANGING slots: level-(l-1) slots of the corners of the
 *                              coarse cell floor(x/3) with a non-zero d-linear weight
 *                              (Sect. 3, rule 2), -1 elsewhere
 *  hang_w        n_slots*2^d   the weights prod_i (r_i/3 or (3-r_i)/3), r = x mod 3; 0 where idx = -1
 *  parent        n_slots       level-(l-1) slot at the same position (x = 0 mod 3), else -1
 *                              (the injection I of Sect. 3, rule 1)
 *  child         n_slots       level-(l+1) slot at position 3x, else -1
 *  brick_roots   n_bricks*d    root-cell coordinates on level l-m, in Peano order
 *  brick_nbr     n_bricks*3^d  brick index at root offset o, -1 if none */
mg_status mg_grid_tables(const mg_grid* grid, int level, int32_t* coords, uint8_t* vflags, uint8_t* cflags,
                         int32_t* nbr, int32_t* cell_vertices, int32_t* hang_idx, double* hang_w,
                         int32_t* parent, int32_t* child, int32_t* brick_roots, int32_t* brick_nbr);

void mg_destroy_grid(mg_grid* grid);

/* ---------------------------------------------------------------- options */

typedef enum mg_transfer { MG_TRANSFER_DLINEAR = 0, MG_TRANSFER_BOXMG = 1 } mg_transfer;
typedef enum mg_coarse_op { MG_COARSE_REDISC = 0, MG_COARSE_GALERKIN = 1 } mg_coarse_op;
typedef enum mg_precision {
  MG_PREC_FP64 = 0,       /* everything in FP64, deltas stored in FP64 */
  MG_PREC_MIXED_BF16 = 1, /* FP64 iterative refinement around FP32 V-cycles, deltas BF16 + FP32 scale */
  MG_PREC_MIXED_FP16 = 2, /* same with FP16 codes */
  MG_PREC_MIXED_BPA = 3   /* same with the deltas in the paper's bpa byte codec (Sect. 5):
                             per vertex and operator bpa in {0, 2..8} bytes per entry, chosen
                             against mg_options.eps_mf; single hierarchies only (not in
                             batches, the server or the persistent solve) */
} mg_precision;

typedef enum mg_smoother {
  MG_SMOOTH_JACOBI = 0, /* omega-damped point Jacobi (Alg. 1) */
  MG_SMOOTH_BLOCK = 1   /* block Jacobi (Sect. 4.2): per step, gs_sweeps Gauss-Seidel sweeps over the
                           2^d iota vertices of every 3^d patch (vertices inside a cell of the next
                           coarser level, lexicographic within the patch), then omega-damped Jacobi
                           on the other DoFs.  Uniform levels; single hierarchies only */
} mg_smoother;

typedef enum mg_cycle {
  MG_CYCLE_V = 0,        /* multiplicative V(nu1, nu2) cycles (Alg. 1) */
  MG_CYCLE_ADDITIVE = 1, /* additive multigrid (Alg. 2): per traversal, the coarse corrections of the
                            previous traversal prolongated down (d_l += P d_{l-1}, u_l += P d_{l-1},
                            surplus uh_l = u_l - P u_{l-1}), then fine to coarse r_l = b_l - A_l u_l,
                            rh_l = b_l - A_l uh_l, d_l = omega D_l^-1 r_l, u_l += d_l, u_{l-1} = I u_l,
                            b_{l-1} = R rh_l; every level smoothed, none solved.  FP64 uniform
                            hierarchies, single problems only; mg_solve stops on ||b - A u||_2 */
  MG_CYCLE_BPX = 2       /* BPX (Alg. 3): the additive traversal, except that above the coarsest level
                            the c-points (every coordinate a multiple of 3) skip their own update, which
                            is injected to the coarser level (i_{l-1} = I d_l) and zeroed; the descent
                            applies P d_{l-1} at c-points and P d_{l-1} - P i_{l-1} elsewhere; the coarse
                            iterates are not overwritten by injection.  Same restrictions as additive */
} mg_cycle;

typedef struct mg_options {
  int32_t transfer;       /* mg_transfer (Sect. 4.4: BoxMG, or d-linear) */
  int32_t coarse;         /* mg_coarse_op (Sect. 4.3: Galerkin R A P, or rediscretisation) */
  int32_t precision;      /* mg_precision */
  int32_t nu1, nu2;       /* pre / post smoothing steps of V(nu1, nu2) (Sect. 4.1) */
  double omega;           /* Jacobi damping (Alg. 1 smoothing update) */
  int32_t coarsest_level; /* level solved directly (FP64 Cholesky), 1 <= c < max_level */
  int32_t inner_cycles;   /* mixed: FP32 V-cycles per refinement step */
  int32_t use_graphs;     /* host-stepped solve: capture cycles in CUDA graphs */
  int32_t persistent;     /* 1: whole solve in one cooperative persistent launch (batches: every
                             step in one persistent launch over a work queue, see
                             mg_batch_create); 0: host-stepped, CUDA-graph-captured cycles
                             (default: on GB300 a dependent graph kernel costs ~0.6 us, a
                             grid-wide barrier ~1.2 us) */
  double eps_mf;          /* MG_PREC_MIXED_BPA: absolute bound on |f_bpa(x) - x| per delta entry
                             (Sect. 5 uses 1e-2, 1e-4, 1e-8); default 1e-4 */
  int32_t smoother;       /* mg_smoother (default MG_SMOOTH_JACOBI); nu1, nu2 count its steps */
  int32_t gs_sweeps;      /* MG_SMOOTH_BLOCK: Gauss-Seidel sweeps per patch and step, 1..64 (default 1) */
  int32_t cycle;          /* mg_cycle (default MG_CYCLE_V); mg_vcycle runs one traversal of it */
  int32_t dynamic_coarsest; /* 1: the dynamic coarsest level of Sect. 4.3 (uniform grids, single
                             hierarchies; default 0).  mg_setup audits every coarse level: a level
                             with a DoF row whose diagonal is not positive or whose off-diagonal
                             magnitudes over the unknowns exceed the diagonal (beyond a relative
                             1e-12) makes the level above it the coarsest one; mg_solve (FP64)
                             raises the coarsest level by one after a cycle that reduces the
                             residual by less than a factor 1/0.95.  The coarsest level stays at
                             most 1024 unknowns (it is solved directly): a raise beyond that, or to
                             the finest level, makes mg_setup return MG_ERR_INDEFINITE_COARSE.
                             mg_get_coarsest reports the level in use */
  int32_t tensor_coefficients; /* 1: the hierarchy takes diagonal-tensor coefficients eps = diag(eps_i)
                             through mg_setup_tensor (the paper's `checkerboard` benchmark, Sect. 7;
                             default 0).  Uniform grids, Galerkin coarse operators, Jacobi smoother,
                             single hierarchies (not batches, the server, the persistent solve or
                             the bpa codec) */
  int32_t ff_sweeps;      /* 1: the finest level's Jacobi and residual sweeps of an FP64 hierarchy run
                             in float-float arithmetic (value = h + l of two binary32 numbers,
                             error-free TwoSum / TwoProduct; GB300's FP64 units run at ~1/64 of its
                             FP32 rate).  Vectors and the setup stay binary64; a sweep result
                             differs from FP64 arithmetic by a few 2^-47 (instead of 2^-53) of the
                             sum of its absolute terms, so mg_smooth, mg_residual and mg_vcycle
                             return float-float results.  mg_solve runs float-float cycles while
                             the relative residual exceeds 1000 x rel_tol (or until a cycle reduces
                             it by less than 5%), then FP64 cycles: the solution carries the FP64
                             residual floor (float-float alone stalls ~2^6 higher: near 1e-10 on
                             the 2D level-6 1:1e-4 checkerboard).  Nonzero |values| must lie in
                             [2^-103, 2^127): smaller ones count as zero, larger ones give NaN (a
                             non-finite residual).  Single FP64 hierarchies with the Jacobi smoother
                             and V-cycles, 2D and 3D (host-stepped solves; batches, the server and
                             the persistent solve keep FP64 sweeps); default 0 */
} mg_options;

void mg_default_options(mg_options* opt); /* BoxMG, Galerkin, FP64, V(2,2), omega 0.6, coarsest 1, eps_mf 1e-4,
                                             Jacobi smoother */

/* ---------------------------------------------------------------- hierarchy */

/* Allocate the device-resident hierarchy of a grid (operators, deltas, work
 * vectors) on the current device.  Allocation happens here only.
 * Adaptive grids (Sect. 3, hierarchical generating system): a grid whose levels
 * 0 .. L-2 are refined everywhere, so that level t = L-1 is complete and only its
 * refinement to level L is partial, gets a composite hierarchy: BoxMG / Galerkin
 * operators on the complete levels t .. c, d-linear transfer between t and L, and
 * the composite cycle of mg_vcycle / mg_solve.  Needs coarsest_level < L-1.
 * Errors: MG_ERR_INVALID_ARG, MG_ERR_OOM, MG_ERR_UNSUPPORTED (an adaptive grid
 * refined in part below level L-1). */
mg_status mg_hier_create(const mg_grid* grid, const mg_options* opt, mg_hier** out);

/* Device bytes mg_hier_create would allocate for this grid and options (admission
 * control and capacity planning).  opt NULL = defaults. */
mg_status mg_hier_footprint(const mg_grid* grid, const mg_options* opt, size_t* bytes);

/* Setup (A8-A11): from leaf-cell coefficients eps (device, level-concatenated cell
 * slots, n = sum of n_slots over levels 0..L, read at existing unrefined cells),
 * compute coarse coefficients (mean of the 3^d children), BoxMG P per coarse
 * vertex (App. C: one C(s) p = f solve per patch corner), Galerkin A_{l-1} =
 * R A_l P with R = P^T (Sect. 4.3), the hierarchical deltas A_hat, P_hat
 * (Sect. 5), their BF16/FP16 codes or bpa byte streams for the mixed path, and the
 * FP64 Cholesky factor of the coarsest operator.  Enqueued on stream.
 * Errors: MG_ERR_INDEFINITE_COARSE if a coarse stencil has a non-positive
 * diagonal or the coarsest Cholesky fails (Sect. 4.3 definiteness check);
 * MG_ERR_NONFINITE if a delta cannot be stored in the bpa codec. */
mg_status mg_setup(mg_hier* h, const double* eps, void* stream);

/* Setup for a diagonal-tensor coefficient eps = diag(eps_1, .., eps_d) per leaf cell
 * (eq. "pde" with a diagonal diffusion tensor; the paper's `checkerboard` benchmark,
 * Sect. 7, Table "parameters"), for hierarchies created with tensor_coefficients = 1.
 * eps_axes: device, d level-concatenated cell arrays one after the other (axis i at
 * eps_axes + i * n, n = sum of n_slots over levels 0..L, layout as mg_setup's eps).
 * The finest level's stencils are rebuilt in situ from the per-cell mean of eps_i plus
 * the anisotropic part (per pair of corners, 2D: -d_x/2 for corners differing in x only,
 * +d_x/2 for those differing in y only; 3D, times h: -d_i/6 along axis i, +d_k/12 for
 * corners differing in the two axes other than k; d_i = eps_i - mean), applied by a
 * correction pass after every finest-level sweep; coarse levels carry the anisotropy in
 * their Galerkin operators (A_hat).  mg_setup on such a hierarchy sets eps_i = eps for
 * all i.  Errors as mg_setup. */
mg_status mg_setup_tensor(mg_hier* h, const double* eps_axes, void* stream);

/* ---------------------------------------------------------------- A3-A7 steps (FP64) */

/* nu smoothing steps of the hierarchy's smoother on level, in place on u (device,
 * n_slots); b device, n_slots.  MG_SMOOTH_JACOBI: damped Jacobi sweeps
 * u <- u + omega diag(A)^-1 (b - A u) (Alg. 1); MG_SMOOTH_BLOCK: block Jacobi steps
 * (Sect. 4.2, see mg_smoother). */
mg_status mg_smooth(mg_hier* h, int level, double* u, const double* b, int nu, void* stream);

/* r = b - A u on level (device vectors).  norm2_host (nullable): receives
 * sum over DoFs of r^2, computed by a fixed-order reduction; non-NULL
 * synchronises the stream. */
mg_status mg_residual(mg_hier* h, int level, const double* u, const double* b, double* r,
                      double* norm2_host, void* stream);

/* b_coarse = R r_fine, R = P^T (Sect. 4.4), from fine_level to fine_level-1. */
mg_status mg_restrict(mg_hier* h, int fine_level, const double* r_fine, double* b_coarse, void* stream);

/* u_fine += P e_coarse (Alg. 1 coarse-grid correction), fine_level-1 -> fine_level. */
mg_status mg_prolong(mg_hier* h, int fine_level, const double* e_coarse, double* u_fine, void* stream);

/* u on HANGING slots of level <- d-linear interpolant of level-1 (Sect. 3, rule 2). */
mg_status mg_interpolate_hanging(mg_hier* h, int level, const double* u_coarse, double* u_fine, void* stream);

/* FP32 counterparts on a mixed-precision hierarchy (the inner solver of the mixed
 * path): same operations in FP32 arithmetic, coarse-level deltas decoded from
 * their BF16/FP16 codes times the per-vertex FP32 scale, coefficients rounded to
 * FP32.  u, b, r: device float vectors of n_slots.  MG_ERR_INVALID_ARG on an FP64
 * hierarchy. */
mg_status mg_smooth_f32(mg_hier* h, int level, float* u, const float* b, int nu, void* stream);
mg_status mg_residual_f32(mg_hier* h, int level, const float* u, const float* b, float* r, double* norm2_host,
                          void* stream);
mg_status mg_vcycle_f32(mg_hier* h, float* u, const float* b, void* stream); /* uniform grids only */

/* Allocation-free residual: r = b - A u on level and the squared norm of r over the
 * DoFs, written to the device double *norm2 (no host copy, no synchronisation).
 * The paper has no counterpart; this is a service of the library for callers that
 * must not call cudaMalloc: code running under a fixed device-memory budget handed
 * out by a host framework, or latency-critical loops where an allocation call could
 * block on work already queued on the GPU.  The hierarchy h is created beforehand.
 * The reduction's per-CTA partial sums live in a file-scope device array of 4096
 * doubles (32 KiB, held by every GPU that loads the library until the process
 * exits); a level whose sweep needs more than 4096 per-CTA partial sums (bricks x
 * slabs) is rejected with MG_ERR_INVALID_ARG (2D up to level 6 and 3D up to level 4
 * fit).  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress) with the device current;
 * make that first call before any stream capture.  Every call on a device shares
 * the one array, so calls whose kernels overlap on the GPU (concurrent streams)
 * race; serialise them.  *norm2 agrees with mg_residual's norm to about 1e-15
 * relative (the partial sums are added with another stride), not bit for bit.  The
 * finest level of a tensor-coefficient hierarchy is rejected (MG_ERR_UNSUPPORTED).
 * u, b, r: device vectors of n_slots; norm2: device. */
mg_status mg_residual_norm_noalloc(mg_hier* h, int level, const double* u, const double* b, double* r,
                                   double* norm2, void* stream);

/* Tile autotuner (A13): for every level, time the smoother with each slab depth R
 * dividing the brick edge (B, B/3, ..., 1 planes per CTA) on the level's own buffers
 * and keep the fastest for later sweeps of this hierarchy (FP64 sweeps; FP32 sweeps on
 * a mixed hierarchy).  Results are unchanged by the choice (every vertex is computed by
 * the same arithmetic); only the split of work over CTAs differs.  chosen (host,
 * nullable, 2 * (max_level + 1) ints): [2l] the FP64 and [2l+1] the FP32 depth of
 * level l (0 where not tuned).  Call after mg_setup; synchronises stream. */
mg_status mg_autotune(mg_hier* h, int32_t* chosen, void* stream);

/* ---------------------------------------------------------------- A12 cycles */

/* One V(nu1, nu2) cycle on the finest level (correction scheme; on uniform
 * grids with Galerkin coarse operators this is the FAS/HTMG cycle of Sect. 3 /
 * Alg. 1).  u, b device finest-level vectors; u updated in place. FP64.
 * Adaptive hierarchy: one composite cycle (Sect. 3: FAS on the levels t = L-1 and
 * L; nu1 Jacobi sweeps on level L with hanging values interpolated from level t,
 * the level-t correction equation with R r_L at refined and the level-t residual
 * at unrefined vertices solved by one V-cycle of levels t .. c, d-linear
 * correction of level L, nu2 sweeps).  u and b are then level-concatenated vectors
 * (slot_offset / n_slots of mg_grid_info, like eps); only the level-L and level-t
 * segments are read or written.  The unknowns are the level-L DoFs and the
 * unrefined level-t DoFs; b is read there only.  On return the level-L hanging
 * entries hold the interpolant of level t and the refined level-t entries the
 * injected level-L value (Sect. 3, rules 1 and 2); on entry the hanging entries
 * are recomputed and every other non-unknown entry must be zero.
 * Additive hierarchy (MG_CYCLE_ADDITIVE): one traversal of Alg. 2 instead, on the
 * coarse iterates and corrections the hierarchy keeps between calls (zeroed by
 * mg_setup and at the start of mg_solve). */
mg_status mg_vcycle(mg_hier* h, double* u, const double* b, void* stream);

typedef struct mg_solve_stats {
  int32_t cycles;          /* V-cycles run (mixed: FP32 inner cycles) */
  int32_t outer_steps;     /* mixed: FP64 refinement steps; FP64: = cycles */
  double rel_residual;     /* final ||r||_2 / ||r_0||_2 (FP64 residual) */
  double r0_norm;          /* ||b - A u_0||_2 */
  double solve_ms;         /* wall time of the call */
  double* history;         /* host, nullable: per-check relative residuals */
  int32_t history_capacity;
  int32_t history_len;
} mg_solve_stats;

/* Solve A u = b from u = 0 on the finest level until ||r||/||r0|| <= rel_tol
 * (Euclidean over DoFs) or max_cycles.  FP64: V-cycles (additive hierarchies:
 * traversals of Alg. 2, counted as cycles).  Mixed: FP64 residual and update
 * (iterative refinement) around inner_cycles FP32 V-cycles that read the
 * BF16/FP16 codes or the bpa streams of the deltas.  The block smoother, where
 * chosen, replaces the Jacobi sweeps of every cycle.  u, b device; stats host,
 * nullable.  Synchronises stream.
 * Returns MG_ERR_NOT_CONVERGED / MG_ERR_DIVERGED / MG_ERR_NONFINITE with u holding
 * the last iterate.  Adaptive hierarchy: composite cycles on level-concatenated u
 * and b (layout as in mg_vcycle); the residual is the composite one (level-L DoFs
 * and unrefined level-t DoFs); the mixed path refines both levels in FP64 around
 * FP32 composite cycles; `persistent` is ignored. */
mg_status mg_solve(mg_hier* h, double* u, const double* b, double rel_tol, int max_cycles,
                   mg_solve_stats* stats, void* stream);

/* ---------------------------------------------------------------- A13 batched solves */

typedef struct mg_batch mg_batch;

/* Group n set-up hierarchies (same dimension and options, any sizes) into one batch.
 * The problems of a batch advance through their V-cycles in lockstep, aligned by
 * depth below their own finest level; every phase of a cycle is one launch per brick
 * edge over the work items of all problems.  With options.persistent = 1 on every
 * hierarchy (BoxMG + Galerkin with BF16 codes, or geometric hierarchies), every step
 * (an FP64 cycle, or a mixed refinement step with its inner cycles) is instead one
 * persistent launch over a device work queue of the problems' items in phase order,
 * each problem advancing by its own progress counter; a wait that runs out makes
 * mg_batch_solve return MG_ERR_TIMEOUT.  hiers: host array of n handles that must
 * outlive the batch (the batch reads their operators; re-running mg_setup on them
 * keeps the batch valid).  Errors: MG_ERR_INVALID_ARG on mismatched options or
 * hierarchies not set up (or with more than 64 coarsest DoFs). */
mg_status mg_batch_create(int n, mg_hier* const* hiers, mg_batch** out);

/* mg_setup of every problem of the batch (eps: host array of n device pointers, as in
 * mg_setup), enqueued back to back with one synchronisation and one status check at
 * the end instead of one per problem.  Errors as mg_setup (the first failing problem). */
mg_status mg_batch_setup(mg_batch* batch, const double* const* eps, void* stream);

/* Solve all problems of the batch from u = 0 to rel_tol each (FP64, or FP64
 * refinement around inner_cycles FP32 V-cycles for mixed hierarchies).  u, b: host
 * arrays of n device pointers (finest-level vectors of each problem).  stats: host
 * array of n entries (nullable); per-problem cycles, r0, final relative residual,
 * status.  Converged problems retire on the device while the others continue.
 * Synchronises the stream.  Returns the first non-OK per-problem status. */
mg_status mg_batch_solve(mg_batch* batch, double* const* u, const double* const* b, double rel_tol, int max_cycles,
                         mg_solve_stats* stats, void* stream);

void mg_batch_destroy(mg_batch* batch);

/* ---------------------------------------------------------------- A13 serving */

typedef struct mg_server mg_server;

typedef struct mg_request {
  const mg_grid* grid; /* uniform grid of the problem (caller-owned, alive until done) */
  const double* eps;   /* device, level-concatenated leaf coefficients (as mg_setup) */
  const double* b;     /* device, finest-level right-hand side */
  double* u;           /* device, finest-level solution (written by the server) */
  double rel_tol;
  int32_t max_cycles;
  int32_t reserved;
} mg_request;

/* Start a server on the current device: it admits queued requests whose hierarchies
 * fit the rest of hbm_budget_bytes (scanning in arrival order; a request that does not
 * fit yet does not hold back later ones that do), sets them up, and runs the admitted
 * requests in three lanes by finest-level size (under 2^16 DoFs, under 2^20, larger),
 * each a continuously re-formed batch on its own stream and thread, the smaller lanes at
 * higher stream priority (requests join at their lane's next step boundary and retire,
 * releasing their memory, as soon as they converge).  opt: options of every request
 * (NULL = defaults; options.persistent = 1 runs the lanes' steps as persistent
 * launches). */
mg_status mg_server_create(size_t hbm_budget_bytes, const mg_options* opt, mg_server** out);

/* Queue a request; *ticket identifies it.  The request's buffers must stay valid until
 * it is done.  MG_ERR_BUDGET if its hierarchy alone exceeds the budget. */
mg_status mg_server_submit(mg_server* server, const mg_request* req, uint64_t* ticket);

/* *done = 1 once the request finished (then stats, nullable, get its cycles, r0,
 * final relative residual and latency from submission in solve_ms, and the ticket is
 * released); wait != 0 blocks until then.  Returns the request's status when done. */
mg_status mg_server_poll(mg_server* server, uint64_t ticket, int wait, int* done, mg_solve_stats* stats);

/* Queue length, running requests and device bytes held by admitted requests. */
mg_status mg_server_info(mg_server* server, int64_t* queued, int64_t* running, size_t* bytes_in_use);

/* Stops the thread (requests still queued or running are abandoned) and frees everything. */
void mg_server_destroy(mg_server* server);

/* ---------------------------------------------------------------- inspection (parity tests) */

/* Reconstructed FP64 operator stencils of a level, A_redisc + A_hat
 * (device, n_slots*3^d, offset-major: st[k*n_slots + slot]). */
mg_status mg_get_stencils(mg_hier* h, int level, double* st, void* stream);

/* FP64 deltas stored for a coarse level (device, nullable, offset-major):
 * a_hat n_slots*3^d (Galerkin), p_hat n_slots*5^d (BoxMG P of level -> level+1,
 * offsets in [-2,2]^d lexicographic). */
mg_status mg_get_deltas(mg_hier* h, int level, double* a_hat, double* p_hat, void* stream);

/* Mixed-path codes and scales of a coarse level (device, nullable, offset-major).
 * a_scale carries the promotion flag of A_hat as its sign bit (see mg_encode_deltas_promote). */
mg_status mg_get_codes(mg_hier* h, int level, uint16_t* a_codes, float* a_scale, uint16_t* p_codes,
                       float* p_scale, void* stream);

/* Low halves of the A_hat codes of a coarse level of a BF16/FP16 hierarchy (device,
 * n_slots*3^d, offset-major): non-zero only on promoted vertices, whose FP32 codes are
 * (a_codes << 16 | a_lo).  MG_ERR_INVALID_ARG on FP64 / bpa hierarchies and the finest level. */
mg_status mg_get_code_lo(mg_hier* h, int level, uint16_t* a_lo, void* stream);

/* Standalone delta encoder (A10): for n rows of k FP64 entries (device, row-major
 * delta[i*k + j]) write scale[i] = fl32(max_j |delta|) and codes = RNE to
 * fmt (1 = BF16, 2 = FP16) of delta / scale formed in FP64 (device outputs). */
mg_status mg_encode_deltas(int64_t n, int k, const double* delta, int fmt, uint16_t* codes, float* scale,
                           void* stream);

/* The same encoder with per-row promotion (A10; the dtype counterpart of the paper's
 * per-vertex storage choice against eps_mf, Sect. 5): reconstructing A = A_redisc + A_hat
 * cancels where the delta is as large as the operator, so a row whose worst 16-bit
 * rounding, h s (h = 2^-9 for BF16, 2^-12 for FP16, s = fl32(max_j |delta|)), exceeds
 * 2^-8 |diag[i]| (diag: the row's reconstructed diagonal A_vv, device, n FP64) is stored
 * as the FP32 bit pattern of fl32(delta / s) (RNE of the FP64 quotient): high half in
 * codes, low half in lo, and scale[i] = -s (the sign bit is the flag).  Other rows:
 * codes as mg_encode_deltas, lo = 0, scale[i] = +s.  Decoding: promoted rows
 * fl32(float(codes << 16 | lo) * s), others fl32(value16(codes) * s).
 * All buffers device, row-major n x k (scale, diag: n). */
mg_status mg_encode_deltas_promote(int64_t n, int k, const double* delta, const double* diag, int fmt,
                                   uint16_t* codes, uint16_t* lo, float* scale, void* stream);

/* The bpa byte codec of Sect. 5 on caller buffers (NEXT row: the paper's delta storage).
 * Each of n rows of k FP64 entries (device, row-major x[i*k + j]) is one operator: it is
 * dropped (bpa = 0) if every |entry| <= eps_mf, else stored with the smallest bpa in
 * {2, ..., 8} for which every entry's f_bpa = (-1)^s m 2^e satisfies |f_bpa - x| <= eps_mf.
 * An entry takes bpa bytes: e (int8), then the bpa - 1 bytes of m little-endian, whose top
 * bit is the sign s and whose other 8 (bpa - 1) - 1 bits hold |m|; e is the smallest
 * exponent for which |m| = rint(|x| 2^-e) fits those bits (clamped below at -128).
 * Outputs (device): rec[i] = (byte offset of row i << 4) | bpa_i, rows one after the
 * other in `bytes` (capacity n * k * 8 bytes, the worst case), *total_bytes = the
 * stream's length, *status (nullable) = 0, or 1 if an entry is not finite, 2 if an entry
 * is beyond every bpa's exponent range (those rows are recorded with bpa 0).
 * Enqueued on stream (three launches); k in 1..125. */
mg_status mg_bpa_encode(int64_t n, int32_t k, const double* x, double eps_mf, uint64_t* rec, uint8_t* bytes,
                        uint64_t* total_bytes, int32_t* status, void* stream);

/* Decode rows written by mg_bpa_encode (device buffers): out[i*k + j] = f_bpa of entry j
 * of row i, in FP64 (fp32 = 0, exact) or FP32 (fp32 = 1: |m| rounded once to FP32 and
 * scaled by 2^e, as the FP32 cycle kernels decode).  The decoder reads the stream by
 * aligned 8-byte words: `bytes` must be 8-byte aligned and its buffer a multiple of 8
 * bytes long (the n * k * 8 bytes mg_bpa_encode asks for are). */
mg_status mg_bpa_decode(int64_t n, int32_t k, const uint64_t* rec, const uint8_t* bytes, int32_t fp32, void* out,
                        void* stream);

/* A MG_PREC_MIXED_BPA hierarchy's codec on a coarse level: copies (device, nullable) of
 * the per-slot records and byte streams of A_hat (3^d entries per vertex, plane order)
 * and P_hat (5^d); a_bytes / p_bytes (host, nullable) receive the streams' lengths.
 * Buffers hold n_slots records and n_slots * 3^d * 8 (5^d * 8) bytes.  Synchronises. */
mg_status mg_get_bpa(mg_hier* h, int level, uint64_t* a_rec, uint8_t* a_stream, uint64_t* p_rec, uint8_t* p_stream,
                     uint64_t* a_bytes, uint64_t* p_bytes, void* stream);

/* The level a hierarchy currently solves directly (host *level): the coarsest_level of
 * its options, or the level the dynamic rule (mg_options.dynamic_coarsest) chose. */
mg_status mg_get_coarsest(mg_hier* h, int32_t* level);

void mg_destroy_hier(mg_hier* h);

/* ---------------------------------------------------------------- measurement */

/* FP64 fma-rate probe (the paper has no counterpart: it measures the denominator of
 * the FP64 roofline that bounds the sweeps on this GPU).  Launches n_ctas CTAs of 256
 * threads; every thread runs 8 independent chains of iters dependent FP64 fmas.  Time
 * it with events on `stream`; *flops (host) receives the fma flops of the launch
 * (2 per fma).  sink: device array of n_ctas doubles (never written for these inputs;
 * it keeps the chains from being optimised away).  n_ctas in 1..2^24, iters >= 1,
 * else MG_ERR_INVALID_ARG.  Enqueued only; no synchronisation. */
mg_status mg_probe_fp64_fma(int64_t n_ctas, int32_t iters, double* sink, int64_t* flops, void* stream);

const char* mg_last_error(void);
const char* mg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
