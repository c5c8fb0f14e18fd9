/*
 * coupledmg.h - C ABI of the GB300 multigrid solver for the coupled
 * pressure-temperature Poisson-Helmholtz system of Saade, Lohse & Fuster
 * (arXiv 2206.11294), Sec. 3, Eqs. 27-34.
 *
 * The system (unknown per cell a = (T, p), the paper's order):
 *
 *   div(k grad T)     + l1 T + l2 p                    = lambda_T   (Eq. 27)
 *   div((1/rho) grad p) + l3 p + l4 div(k grad T)      = lambda_p   (Eq. 28)
 *
 * with per-cell l1..l4 (Eqs. 29-32) and right-hand side lambda_T, lambda_p
 * (Eqs. 33-34), discretised with cell-centred finite volumes on a uniform grid
 * (2D Cartesian, 2D axisymmetric (r, z), 3D Cartesian).  It is solved by the
 * paper's defect-correction loop (Sec. 3, the four steps after Eq. 34) with
 * one multigrid V-cycle as the correction solve, entirely on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Cells are numbered x-fastest: id = i + n0*(j + n1*k).
 * - Faces normal to axis a carry n_a + 1 entries along a and n_b along the
 *   other axes, numbered x-fastest in that shape: boundary faces included.
 * - Cell arrays of pairs are [N][2] doubles, (T, p) or (lambda_T, lambda_p);
 *   lambda is [N][4] doubles, l1..l4.
 * - Pointers are host pointers when on_device == 0 and device pointers of the
 *   handle's device when on_device == 1.  Device pointers must be 16-byte
 *   aligned.  The caller owns every buffer it passes; the library copies what
 *   it keeps.
 * - Every call runs on the CUDA stream given to mg_create and returns after
 *   that work has completed (the *_async calls excepted).
 * - Errors are returned as mg_status; no exception or signal crosses the ABI.
 *   mg_last_error() gives a thread-local message for the last failure.
 *   Arguments are validated before any output is written.
 */
#ifndef COUPLEDMG_H
#define COUPLEDMG_H

#include <stddef.h>

#if defined(__GNUC__)
#define MG_API __attribute__((visibility("default")))
#else
#define MG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,     /* bad sizes, kinds, pointers, or a grid whose coarsest level is too large */
    MG_ERR_OOM = 2,             /* device allocation failed */
    MG_ERR_BUDGET = 3,          /* workspace given to mg_create too small */
    MG_ERR_INVALID_COEFF = 4,   /* a local 2x2 block is singular or not finite */
    MG_ERR_NOT_CONVERGED = 5,   /* max_cycles reached; x and stats still written */
    MG_ERR_TIMEOUT = 6,         /* a bounded device-side wait gave up */
    MG_ERR_CUDA = 7,            /* a CUDA runtime call failed (message in mg_last_error) */
    MG_ERR_STATE = 8            /* call out of order (e.g. mg_solve before mg_set_coeffs) */
} mg_status;

/* Boundary kinds per axis and side (Appendix B uses Dirichlet p; Sec. 5.2 a
 * rigid no-flux wall; the axisymmetric runs a symmetry axis at r = 0). */
enum { MG_BC_WALL = 0, MG_BC_DIRICHLET = 1, MG_BC_AXIS = 2 };

/* Precision of the multigrid cycles. */
enum { MG_FP64 = 0, MG_MIXED = 1 };

typedef struct {
    int dim;             /* 2 or 3 */
    int axisym;          /* 1: dim == 2 and axis 0 is the radius r, axis 1 is z */
    int n[3];            /* cells per axis, n[2] = 1 when dim == 2 */
    double h;            /* uniform cell size */
    double r0;           /* axisymmetric: radius of the low-r face (0: the symmetry axis) */
    int bc[3][2];        /* MG_BC_* per axis, low and high side */
    double bc_T[3][2];   /* Dirichlet values of T (used where bc == MG_BC_DIRICHLET) */
    double bc_p[3][2];   /* Dirichlet values of p */
} mg_grid;

typedef struct {
    int nu1, nu2;        /* pre- and post-smoothing sweeps per level (default 2, 2) */
    int precision;       /* MG_FP64 or MG_MIXED (FP32 cycles inside FP64 refinement) */
    double rtol;         /* stop when both per-field norms fell by rtol; <= 0: run max_cycles */
    int max_cycles;      /* FP64: V-cycles; MIXED: outer refinement steps */
    int coarse_min;      /* coarsen while every n_a is even and n_a/2 >= coarse_min (default 4) */
    int inner_cycles;    /* MIXED: FP32 V-cycles per outer step (default 1) */
    int cycle;           /* MG_CYCLE_V (default), MG_CYCLE_W or MG_CYCLE_F: the correction solve's cycle.  W visits
                            each coarser level twice (W, W), F twice (F, then V); the second visit continues from
                            the first one's coarse solution; the exactly solved coarsest level is solved once.  W and
                            F run without the V-cycle tail kernel (mg_tuning.tail_level is ignored); batches take V
                            only. */
    int smoother;        /* MG_SMOOTH_RBGS (default): red-black block Gauss-Seidel, red (even i+j+k) first;
                            MG_SMOOTH_WJAC: weighted block Jacobi, each cell's two rows solved against the
                            previous iterate, then x_i += omega (z_i - x_i).  The paper names a multigrid solver
                            without its smoother (Sec. 3); both give the same fixed point.  WJAC runs one kernel
                            per sweep (mg_tuning.sweep, tile and tail_level are ignored; persistent applies) and
                            batches take RBGS only. */
    double omega;        /* MG_SMOOTH_WJAC: the weight, 0 < omega <= 1 (default 0.8) */
    double fp64_jump_ratio; /* MIXED: a finest-level cell whose interior faces' k or 1/rho differ by more than this
                            ratio (a cell at the bubble interface) has its 2x2 block applied in FP64 inside the
                            FP32 cycles (the FP64 W and Dinv r of the cell; every other cell stays FP32).
                            0: off; otherwise >= 1 (default 2: the interface the volume fraction smooths over
                            about two cells changes the coefficients by up to ~5x per cell there).  Ignored in
                            FP64. */
    int coarse_solve;    /* The exact coarsest solve (Sec. 3 names a direct solve there).  Both factor the
                            coarsest matrix once per mg_set_coeffs (banded LU with partial pivoting, FP64).
                            MG_COARSE_AUTO (default): coarsest systems above 128 unknowns (odd grid factors of 9
                            or more, e.g. 31 x 31 cells for n = 992) keep the factors and each cycle runs the two
                            triangular solves, one warp, 2n dependent steps; smaller ones form the inverse and
                            each cycle multiplies by it.  MG_COARSE_INVERSE: always form the inverse (its n^2
                            (kl + ku) set-up work pays back only over many cycles).  A hierarchy that solves
                            from the factors runs without the V-cycle tail kernel (mg_tuning.tail_level must be
                            >= levels).  Batches need one value for all their handles. */
} mg_options;

enum { MG_CYCLE_V = 0, MG_CYCLE_W = 1, MG_CYCLE_F = 2 };
enum { MG_SMOOTH_RBGS = 0, MG_SMOOTH_WJAC = 1 };
enum { MG_COARSE_AUTO = 0, MG_COARSE_INVERSE = 1 };

typedef struct {
    int cycles;          /* V-cycles run (MIXED: total FP32 cycles) */
    int outer;           /* MIXED: outer FP64 steps; FP64: equals cycles */
    double r0[2];        /* initial per-field stopping norms ||D^-1 r||_2 (T, p) */
    double rfinal[2];    /* final per-field stopping norms */
    double seconds;      /* wall time of the call */
    int status;          /* mg_status of the solve */
    int levels;          /* multigrid levels of the hierarchy */
    long long fp64_cells; /* MIXED: finest-level cells whose 2x2 block the FP32 cycles apply in FP64 */
} mg_stats;

typedef struct mg_handle mg_handle;

/* Fills defaults: V(2,2), FP64, rtol 1e-10, 50 cycles, coarse_min 4, 1 inner cycle, red-black block
 * Gauss-Seidel (omega 0.8 for weighted block Jacobi), FP64 blocks at face-coefficient jumps above 2:1
 * in mixed precision, MG_COARSE_AUTO. */
MG_API mg_status mg_default_options(mg_options *opt);

/* Device bytes a handle of this grid and these options needs (hierarchy,
 * coarse inverse, staging).  No device work. */
MG_API mg_status mg_workspace_size(const mg_grid *grid, const mg_options *opt, size_t *bytes);

/* Creates a solver for one grid on the current CUDA device.
 *   workspace, workspace_bytes: device memory of at least mg_workspace_size
 *     bytes, owned by the caller and kept alive until mg_destroy; NULL lets the
 *     library allocate (and free) its own.
 *   stream: a cudaStream_t (NULL = legacy default stream) for all later work.
 * The handle is not thread-safe; distinct handles may be used concurrently. */
MG_API mg_status mg_create(const mg_grid *grid, const mg_options *opt, void *workspace,
                    size_t workspace_bytes, void *stream, mg_handle **out);

/* Coefficient intake and set-up (Eqs. 27-32): per-cell lambda [N][4] = l1..l4
 * and per-axis face arrays of 1/rho (face_alpha[a]) and k (face_k[a]) for
 * a < dim.  Builds the whole hierarchy on the device: the per-cell 2x2 blocks
 * of Eqs. 27-28, coarse coefficients (area-weighted faces, volume-weighted
 * l1..l4) and the exact coarsest solve.  MG_ERR_INVALID_COEFF if an input is
 * not finite or a local block is singular.  The inverse of the coarsest
 * matrix is still being computed (on a private stream) when this returns;
 * the next mg_solve waits for it and reports a singular coarsest matrix as
 * MG_ERR_INVALID_COEFF.  The caller's arrays are no longer read on return. */
MG_API mg_status mg_set_coeffs(mg_handle *h, const double *lambda, const double *const face_alpha[3],
                        const double *const face_k[3], int on_device);

/* Solves L(x) = rhs: rhs [N][2] = (lambda_T, lambda_p) (Eqs. 33-34); x [N][2]
 * = (T, p), in: initial guess (the paper's a~), out: result.  stats may be
 * NULL.  Returns MG_OK on convergence, MG_ERR_NOT_CONVERGED (x written)
 * after max_cycles. */
MG_API mg_status mg_solve(mg_handle *h, const double *rhs, double *x, int on_device, mg_stats *stats);

/* The solve of mg_solve (Sec. 3, the defect-correction loop after Eq. 34),
 * enqueued on the handle's stream without waiting for it: the stop test runs
 * on the device, between the cycles of one CUDA graph (a loop node whose
 * condition a one-thread kernel sets after each cycle's norms), so the host
 * takes no part until the end.  rhs, x: device pointers (16-byte aligned),
 * as for mg_solve with on_device = 1; x holds the result once the work has
 * completed.  The result and statistics equal mg_solve's bit for bit (the
 * same kernels in the same order).  event: NULL, or a cudaEvent_t recorded on
 * the stream after the solve, so later work on other streams can wait for the
 * result on the device.  Arguments are checked before anything is enqueued;
 * errors found on the device (a singular coarsest matrix, a bounded wait that
 * gave up) are reported by mg_solve_async_stats.  The first call on a handle
 * (and the first after mg_set_tuning, mg_autotune or mg_set_timing) captures
 * the graph.  The caller's rhs must stay valid until the work has completed;
 * the handle is not thread-safe. */
MG_API mg_status mg_solve_async(mg_handle *h, const double *rhs, double *x, void *event);

/* Waits for the handle's last mg_solve_async and reports it as mg_solve would:
 * stats (nullable; seconds = device time of the solve), MG_ERR_NOT_CONVERGED
 * after max_cycles, MG_ERR_STATE when no asynchronous solve is pending. */
MG_API mg_status mg_solve_async_stats(mg_handle *h, mg_stats *stats);

/* y = L(x) (Eqs. 27-28 with the grid's Dirichlet values), all pointers on the
 * given side.  A building block for residual checks: res = b - L(x). */
MG_API mg_status mg_apply(mg_handle *h, const double *x, double *y, int on_device);

/* In place: `sweeps` sweeps of the handle's smoother on the finest level of
 * L(x) = rhs: red-black block Gauss-Seidel (red = even i+j+k first; each
 * cell's two equations solved exactly for (T_i, p_i)), or weighted block
 * Jacobi (every cell from the previous iterate, damped by omega). */
MG_API mg_status mg_smooth(mg_handle *h, const double *rhs, double *x, int sweeps, int on_device);

/* Per-field stopping norms ||D^-1 r||_2 (out[2], host) of x for rhs, where
 * r = rhs - L(x) and D is each cell's 2x2 block of its own (T_i, p_i). */
MG_API mg_status mg_residual_norms(mg_handle *h, const double *rhs, const double *x, int on_device,
                            double out[2]);

/* Instrumentation.  mg_set_timing(h, 1) resets the counters and, from then
 * on, brackets one smoothing pass of the finest level in every cycle (the
 * pre-smoothing, or the post-smoothing when nu1 = 0) with CUDA events on the
 * handle's stream (the cycle graphs are re-captured with the two event
 * nodes when the setting changes); 0 turns that off.  Either call resets the
 * counters.  mg_counters reports, since the last reset:
 *   launches          kernels this handle launched (graph nodes counted per replay)
 *   smooth_ms         device time of the timed finest-level smoothing kernels (timing on)
 *   smooth_launches   how many such kernel launches that time covers
 *   smooth_sweeps     how many red-black sweeps those launches performed
 *   smooth_cells      finest-level cells per sweep */
MG_API mg_status mg_set_timing(mg_handle *h, int enable);
MG_API mg_status mg_counters(const mg_handle *h, long long *launches, double *smooth_ms,
                             long long *smooth_launches, long long *smooth_sweeps, long long *smooth_cells);

/* Kernel choices of a hierarchy, and the autotuner that picks them.  The
 * paper has no counterpart: every choice computes the same result, bit for
 * bit (the same per-cell arithmetic in the same order); only the launch
 * structure differs.
 *   sweep[l]    level l's red-black sweeps: MG_SWEEP_COLOUR (one launch per
 *               colour, in place), MG_SWEEP_COLOUR2 (the same with two rows
 *               per thread, half the blocks) or MG_SWEEP_FUSED (2D grids only: one launch
 *               per sweep on tiles staged in shared memory, the red values of
 *               a one-cell ring recomputed per tile);
 *               or MG_SWEEP_ASYNC (2D only: the fused sweep with every operand
 *               of a tile staged by bulk asynchronous copies completing on an
 *               mbarrier, persistent blocks, the next tiles' copies in flight
 *               while a tile is computed; a tile whose two stages exceed one
 *               block's 227 KB of shared memory is refused, e.g. 64 x 16 FP64);
 *               or MG_SWEEP_FUSED2 (2D only, red-black smoothing with
 *               nu1 / 2 + nu2 / 2 even: each pair of sweeps as one launch on
 *               tiles staged with a 4-cell halo, the red and black values of
 *               shrinking rings recomputed per tile; the level's values move
 *               between its two buffers and are back in place at the end of
 *               each cycle);
 *   tile[l]     fused tile shape, cells: 0 = 64 x 16, 1 = 32 x 16, 2 = 32 x 8;
 *   tail_level  the levels from this one to the coarsest run as one kernel
 *               (smoothing, restriction, coarsest solve, prolongation as
 *               stages separated by barriers, the levels' state in shared
 *               memory); >= levels: none.  Allowed from level 1 when at least
 *               two levels (and at most 12) remain, the level has at most
 *               16384 cells and the state fits 200 KB per thread block;
 *   tail_ctas   thread blocks of that kernel: 1 (one block, block barriers),
 *               8 (a cluster; distributed shared memory, cluster barriers),
 *               or 16 where the device allows non-portable cluster sizes.
 *   persistent  colour sweeps, restriction and prolongation launch one block
 *               per tile (0) or one persistent wave of blocks (SMs x resident
 *               blocks) that walk the tiles (1).
 *   overlap     the kernels of a cycle and of the set-up launch as
 *               programmatic dependents of the kernel before them (1): each
 *               is set up while that kernel drains and waits for it on the
 *               device before it touches memory; 0: plain stream order.
 * Defaults after mg_create: colour sweeps for FP64 cycles, fused 64 x 16 for
 * the FP32 cycles of mixed precision on 2D grids; the tail from the first
 * level below the finest with at most 4096 cells, 8 CTAs; overlap 1.
 * mg_autotune also tries one block. */
#define MG_MAX_LEVELS 32
enum { MG_SWEEP_COLOUR = 1, MG_SWEEP_FUSED = 2, MG_SWEEP_ASYNC = 3, MG_SWEEP_COLOUR2 = 4, MG_SWEEP_FUSED2 = 5 };
typedef struct {
    int levels;                 /* mg_get_tuning: the hierarchy's levels (ignored by mg_set_tuning) */
    int sweep[MG_MAX_LEVELS];
    int tile[MG_MAX_LEVELS];
    int tail_level;
    int tail_ctas;
    int persistent;
    int overlap;
} mg_tuning;

MG_API mg_status mg_get_tuning(const mg_handle *h, mg_tuning *out);
/* MG_ERR_INVALID_ARG (handle unchanged) for a choice outside the rules above. */
MG_API mg_status mg_set_tuning(mg_handle *h, const mg_tuning *t);

/* Measures the choices on the handle's own hierarchy and keeps the fastest:
 * per level, each sweep kernel (and tile shape) as one CUDA graph of `reps`
 * pairs of sweeps (median of five replays); then each allowed tail (none,
 * every allowed first level on 1, 8 or 16 CTAs), with and without persistent
 * waves, then the chosen kernels with and without dependent launches (plain
 * order kept only where it is more than 1% faster), each as a graph of one
 * V-cycle
 * launched 4 * reps + 1 times, each launch timed with CUDA events on the
 * handle's stream and waited for, as the solve does per cycle (median), so
 * the per-launch cost of the graph counts.
 * Needs coefficients (MG_ERR_STATE otherwise); overwrites the hierarchy's
 * scratch state (every level's x, b and right-hand sides), not the
 * coefficients, so the next mg_solve is unaffected.  Cycles run in the
 * handle's precision (FP32 for mixed).  out (nullable) receives the chosen
 * tuning, vcycle_ms (nullable) the chosen V-cycle's median time per launch.
 * Synchronous. */
MG_API mg_status mg_autotune(mg_handle *h, int reps, mg_tuning *out, double *vcycle_ms);

/* Batched solve of many independent problems in one set of launches
 * (uneven sizes, e.g. the many bubble grids of one time step).
 * The problems are handles created and given coefficients as usual; they
 * must share dim, options (nu1, nu2, precision, rtol, max_cycles,
 * inner_cycles), stream and device.  Each V-cycle stage runs as one
 * persistent kernel over every problem's tiles, a whole cycle is one CUDA
 * graph replay, and each problem stops on its own with mg_solve's rule, so
 * its result is the one mg_solve gives.  The batch keeps pointers to the
 * handles: destroy the batch before them. */
typedef struct mg_batch mg_batch;
MG_API mg_status mg_batch_create(int count, mg_handle *const *handles, mg_batch **out);

/* rhs[p], x[p]: per problem, as in mg_solve (x in: initial guess, out:
 * result); stats: NULL or count entries.  MG_ERR_NOT_CONVERGED if any
 * problem reached max_cycles (all x and stats still written). */
MG_API mg_status mg_batch_solve(mg_batch *b, const double *const *rhs, double *const *x, int on_device,
                                mg_stats *stats);

/* Coefficient intake and set-up of every problem of the batch in one set of
 * launches (as mg_set_coeffs, per problem): lambda[p] [N_p][4];
 * face_alpha[3*p + a], face_k[3*p + a] the face arrays of problem p, axis a
 * (a < dim).  MG_ERR_INVALID_COEFF names the first failing problem. */
MG_API mg_status mg_batch_set_coeffs(mg_batch *b, const double *const *lambda, const double *const *face_alpha,
                                     const double *const *face_k, int on_device);

/* Kernels launched by this batch since creation (graph nodes per replay). */
MG_API mg_status mg_batch_counters(const mg_batch *b, long long *launches);

/* Kernel choices of a batch (no counterpart in the paper; results are the
 * same, bit for bit, for every choice):
 *   sweep[d], tile[d]  the sweeps of every problem's level d, as mg_tuning's;
 *   blocks_per_sm      persistent grid of every batched kernel: at most this
 *                      many blocks per SM (1..32), each looping over the
 *                      stage's table of (problem, tile) entries.
 * Defaults: fused 64 x 16 for the FP32 cycles of mixed precision in 2D,
 * colour otherwise; 8 blocks per SM.  mg_batch_autotune measures, over all
 * problems at once, each sweep choice per depth (`reps` pairs of sweeps) and
 * then each grid size (`reps` V-cycles), each captured as a CUDA graph and
 * timed with CUDA events (best of three), and keeps the fastest.  Needs the
 * problems' coefficients (MG_ERR_STATE); overwrites scratch state only.
 * out and cycle_ms (time of one V-cycle of the whole batch) are nullable. */
typedef struct {
    int depths;                 /* mg_batch_get_tuning: levels of the deepest problem */
    int sweep[MG_MAX_LEVELS];
    int tile[MG_MAX_LEVELS];
    int blocks_per_sm;
} mg_batch_tuning;

MG_API mg_status mg_batch_get_tuning(const mg_batch *b, mg_batch_tuning *out);
MG_API mg_status mg_batch_set_tuning(mg_batch *b, const mg_batch_tuning *t);
MG_API mg_status mg_batch_autotune(mg_batch *b, int reps, mg_batch_tuning *out, double *cycle_ms);

MG_API mg_status mg_batch_destroy(mg_batch *b);

/* ---------------------------------------------------------------------
 * The steps on either side of the solve (Sec. 3, Algorithm 1): the
 * coefficients of Eqs. 27-34 from the advected state of a time step, and the
 * velocity and phase-pressure update from its solution.  All arrays are
 * device pointers of the current device (host pointers are rejected with
 * MG_ERR_INVALID_ARG), cells and faces in the layouts above; [N][2] and
 * [N][4] arrays 16-byte aligned.  Arguments are validated before anything is
 * launched; the work is then enqueued on `stream` (a cudaStream_t, NULL =
 * legacy default) and the call returns without waiting for it: later work on
 * the same stream (mg_set_coeffs, mg_solve on a handle created with that
 * stream) sees its results.  Inputs are not checked for finiteness
 * (mg_set_coeffs checks what it receives).
 * ------------------------------------------------------------------------- */
typedef struct {
    double Gamma, Pi, b, q;   /* NASG parameters of Eq. 9 (Table 1); ideal gas: Gamma = gamma, Pi = b = q = 0 */
    double cp, cv;            /* heat capacities at constant pressure and volume, J/(kg K), cp > cv > 0 */
    double k;                 /* thermal conductivity, W/(m K), >= 0 */
    double mu;                /* dynamic viscosity, Pa s, >= 0 (read by mg_energy_async only) */
} mg_phase;

typedef struct {              /* the advected state (Eq. Yadv) */
    const double *C;          /* [N] volume fraction of phase 1, in [0, 1] */
    const double *m1, *m2;    /* [N] partial densities C rho_1 and (1 - C) rho_2, kg/m^3 */
    const double *E;          /* [N] averaged total energy per volume, sum of C_i rho_i e_T,i, J/m^3 */
    const double *mom[3];     /* [N] averaged momentum, axes a < dim */
    const double *uf[3];      /* face-normal velocity u* (Eq. provel) on the faces of axis a < dim */
} mg_state;

typedef struct {              /* what mg_set_coeffs and mg_solve take */
    double *lambda;           /* [N][4] lambda_1..lambda_4 (Eqs. 29-32) */
    double *rhs;              /* [N][2] (lambda_T, lambda_p) (Eqs. 33-34) */
    double *x0;               /* [N][2] (T^(adv), p^(adv)), the initial guess; may be NULL */
    double *face_alpha[3];    /* 1/rho on the faces of axis a < dim */
    double *face_k[3];        /* k on the faces of axis a < dim */
} mg_assembly;

/* Coefficient assembly.  Per cell, with C_1 = C, C_2 = 1 - C and overlines
 * the C_i-weighted averages of the phase expressions:
 *   p^(adv) from the averaged total energy minus the kinetic energy
 *     |rho u|^2 / (2 rho), rho = m1 + m2, by the mixture's NASG EOS (Eq. 20);
 *   T^(adv) from p^(adv) (Eq. 23);
 *   beta_i (Eq. 10) and c_i^2 (Eq. 11) at (T^(adv), p^(adv)), rho_i = m_i / C_i;
 *   lambda_1 = -(m1 cp1 + m2 cp2) / dt, lambda_2 = beta T / dt,
 *   lambda_3 = -bracket / dt^2 with bracket the average of
 *     gamma_i / (rho_i c_i^2) - beta_i^2 T / (rho_i cp_i), gamma_i = cp_i / cv_i,
 *   lambda_4 = average of beta_i / (rho_i cp_i), divided by dt unless flags
 *     has MG_ASSEMBLE_LAMBDA4_PRINTED (Eq. 32 as printed lacks the 1/dt that
 *     dividing Eq. 19 by dt gives),
 *   lambda_T = lambda_1 T + lambda_2 p, lambda_p = lambda_3 p + div(u*) / dt,
 *     div the finite-volume divergence (r_f / r_i on axisymmetric r-faces);
 *   faces: 1/rho_f with rho_f the mean of the two cells' rho, k_f = C_f k1 +
 *     (1 - C_f) k2 with C_f the mean of their C, or with MG_ASSEMBLE_HARMONIC_K
 *     the series mean 2 k_L k_R / (k_L + k_R) of the cells' k = C k1 + (1 - C) k2
 *     (conduction through the two half cells); a boundary face takes its cell's.
 * A phase with C_i = 0 in a cell contributes nothing there.  dt > 0. */
enum { MG_ASSEMBLE_LAMBDA4_PRINTED = 1, MG_ASSEMBLE_HARMONIC_K = 2 };
MG_API mg_status mg_assemble_async(const mg_grid *grid, const mg_phase phases[2], double dt, int flags,
                                   const mg_state *state, const mg_assembly *out, void *stream);

/* Update after the solve.  x [N][2] is the solution (T, p) of mg_solve;
 * face_alpha the faces' 1/rho (from mg_assemble_async); uf_star the u* of the state.
 *   uf_out[a] = uf_star[a] - dt face_alpha[a] (grad p)_f  (Eq. unp1 at the
 *     faces), with (p_R - p_L)/h inside, 2 (g - p)/h towards a Dirichlet value
 *     g of grid->bc_p, and 0 at walls and the axis - the face gradients of the
 *     solve's operator, so div uf_out = div u* - dt div((1/rho) grad p);
 *   p1 = p + (1 - C) sigma kappa, p2 = p - C sigma kappa (Eqs. 37-38).
 * uf_out may equal uf_star (in place). */
MG_API mg_status mg_correct_async(const mg_grid *grid, double dt, double sigma, const double *x, const double *C,
                                  const double *kappa, const double *const face_alpha[3],
                                  const double *const uf_star[3], double *const uf_out[3], double *p1, double *p2,
                                  void *stream);

/* Phase energies at the end of the step (Eq. 39):
 *   E_i_out = E_i + dt C_i div F_i,  C_1 = C, C_2 = 1 - C,
 * with the face flux of axis a
 *   F_i = -p_i,f u_f + mu_i (S . u)_{a,f} + k_i (dT/dx_a)_f,  S = grad u + grad u^T,
 * u_f the face velocity uf[a] (u^{n+1} from mg_correct_async), T the first
 * component of x [N][2] (the solution of mg_solve), p1, p2 the phase pressures
 * (from mg_correct_async), E1, E2 the advected phase energies C_i rho_i e_T,i
 * per volume.  A cell's velocity is the mean of its two face velocities; on a
 * face the tangential velocities and p_i are the means of the two cells, normal
 * derivatives the difference across the face, tangential derivatives the mean
 * of the two cells' central differences (one-sided in the first and last cell).
 * Walls and the axis carry no flux; a Dirichlet face carries
 * -bc_p u_f + k_i 2 (bc_T - T)/h towards the boundary value, and no viscous
 * flux.  div is the finite-volume divergence (r_f / r_i on axisymmetric
 * r-faces).  Each face flux is one value shared by its two cells, so the update
 * is conservative to rounding.  E1_out may equal E1 and E2_out E2 (in place);
 * no other output may alias an input.  dt > 0. */
MG_API mg_status mg_energy_async(const mg_grid *grid, const mg_phase phases[2], double dt, const double *x,
                                 const double *C, const double *p1, const double *p2, const double *const uf[3],
                                 const double *E1, const double *E2, double *E1_out, double *E2_out, void *stream);

/* ---------------------------------------------------------------------
 * The implicit momentum predictor (Sec. 3, the equation before Eq. unp1):
 *   (rho/dt) u - div(mu (grad u + grad u^T)) = R
 * for the cell-centred velocity u (dim components), with rho and mu the
 * cells' averaged density and viscosity and R = (rho u)^(adv)/dt - grad p^n +
 * sigma kappa grad C^{n+1} as the caller forms it.  No bulk viscosity
 * (Stokes' hypothesis, Sec. 2).  Discretisation, in finite volumes on the
 * grid of the pressure-temperature solve:
 *   face stress tau_{ca} = mu_f ((du_c/dx_a)_f + (du_a/dx_c)_f), mu_f the mean
 *     of the two cells' mu; normal derivatives across the face, tangential
 *     ones the mean of the two cells' central differences (one-sided in the
 *     first and last cell);
 *   walls (MG_BC_WALL): the normal component is zero on the wall (stress
 *     2 mu 2u/h towards it); tangential components slip freely (no shear), or
 *     with MG_MOMENTUM_NO_SLIP are zero on the wall too (shear mu 2u/h);
 *   pressure boundaries (MG_BC_DIRICHLET) and the axis: no stress;
 *   axisymmetric: r-face stresses weighted by r_f / r_i, and the hoop term
 *     2 mu u_r / r^2 in the r-row.
 * Solution: defect correction on the full residual r = R - A(u); each step
 * solves the component-diagonal part of A (mu weighted 2x on the faces normal
 * to a component) with the pair multigrid of this library, (u_x, u_y) in one
 * hierarchy and, in 3D, u_z in a second.  When the set-up finds the Jacobi
 * bound nu = max over rows of 2 (sum of the component-diagonal operator's
 * off-diagonal entries) / diagonal at most 0.01 (the viscous diffusion number
 * is small: the mass term rho/dt dominates), each step is instead a
 * point-Jacobi step, which contracts the residual at least by nu, and no
 * hierarchy is set up.  Stopping norm ||dt r / rho||_2 over all components and
 * cells.
 * All arrays are device pointers of the handle's device; u, R, y are per
 * component, [N] each (cells in the layout above).  Not thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct mg_momentum mg_momentum;

typedef struct {
    int iterations;           /* outer defect-correction steps */
    int cycles;               /* multigrid cycles of the correction solves, in total */
    double r0, rfinal;        /* stopping norm ||dt r / rho||_2 at the start and at the end */
    double seconds;           /* wall time of the call */
    int status;               /* mg_status of the solve */
    int jacobi;               /* 1: the corrections were point-Jacobi steps, 0: multigrid */
    double nu;                /* Jacobi bound of the set-up: max over rows of 2 (off-diagonal sum) / diagonal */
} mg_momentum_stats;

/* MG_MOMENTUM_MULTIGRID: multigrid corrections whatever the Jacobi bound.
 * MG_MOMENTUM_KRYLOV: with multigrid corrections, restarted GMRES(16)
 *   right-preconditioned by the correction solve, in the inner product of the
 *   stopping norm (iterations then counts GMRES steps); for viscosity-dominated
 *   systems, where plain defect correction contracts by only ~0.5-0.8 per step.
 *   Allocates 17 + 1 vectors of dim N doubles at creation. */
enum { MG_MOMENTUM_NO_SLIP = 1, MG_MOMENTUM_MULTIGRID = 2, MG_MOMENTUM_KRYLOV = 4 };

/* grid: as for mg_create; flags: any of MG_MOMENTUM_NO_SLIP,
 * MG_MOMENTUM_MULTIGRID, MG_MOMENTUM_KRYLOV.  inner: options of
 * the correction solves (NULL: library defaults with one cycle per step);
 * precision must be MG_FP64, rtol is ignored and max_cycles is the number of
 * cycles per correction (run from zero, without stopping norms).  stream: a
 * cudaStream_t for all work. */
MG_API mg_status mg_momentum_create(const mg_grid *grid, int flags, const mg_options *inner, void *stream,
                                    mg_momentum **out);

/* Coefficient intake and set-up of the correction hierarchies: rho, mu [N]
 * (> 0 and >= 0 for a meaningful system; checked only for finiteness through
 * the hierarchies' set-up: MG_ERR_INVALID_COEFF), dt > 0.  The caller's arrays
 * are copied and no longer read on return. */
MG_API mg_status mg_momentum_set_coeffs(mg_momentum *m, double dt, const double *rho, const double *mu);

/* y = A(u), synchronous.  y must not alias u. */
MG_API mg_status mg_momentum_apply(mg_momentum *m, const double *const u[3], double *const y[3]);

/* Solves A u = R; u in: initial guess, out: solution.  Stops when
 * ||dt r/rho|| <= rtol ||dt r0/rho|| (rtol <= 0: runs max_iters steps) or
 * after max_iters steps (MG_ERR_NOT_CONVERGED when rtol > 0; u and stats are
 * still written).  R must not alias u.  stats may be NULL.  MG_ERR_STATE
 * before a successful mg_momentum_set_coeffs. */
MG_API mg_status mg_momentum_solve(mg_momentum *m, const double *const R[3], double *const u[3], double rtol,
                                   int max_iters, mg_momentum_stats *stats);

MG_API mg_status mg_momentum_destroy(mg_momentum *m);

/* The steps either side of the predictor, enqueued on `stream` without
 * waiting (device pointers of the current device, as for mg_assemble_async).
 * Cell gradients are the means of a cell's two face gradients along each
 * axis, the face gradients being those of the projection: (s_R - s_L)/h
 * inside; for p, 2 (g - p)/h towards a Dirichlet value g of grid->bc_p and 0
 * at walls and the axis; for C, 0 at every boundary.
 *
 * Right-hand side: R_c = mom_c / dt - (dp/dx_c) + sigma kappa (dC/dx_c), with
 * mom the advected momentum (rho u)^(adv), p the pressure p^n of the last
 * step, C the volume fraction and kappa the curvature at the new time level.
 * R[a] may equal mom[a] (in place); R must not alias p, C or kappa. */
MG_API mg_status mg_momentum_rhs_async(const mg_grid *grid, double dt, double sigma, const double *const mom[3],
                                       const double *p, const double *kappa, const double *C, double *const R[3],
                                       void *stream);

/* Eq. provel: u* = u_pred + (dt/rho) grad p^n at the cells, and its
 * face-normal components for the projection (the u* that mg_assemble_async
 * and mg_correct_async take): the mean of the two cells' values inside, 0 at
 * walls and the axis, the cell's value at a pressure (Dirichlet) boundary.
 * uf_out must not alias rho, p or u_pred. */
MG_API mg_status mg_provisional_async(const mg_grid *grid, double dt, const double *rho, const double *p,
                                      const double *const u_pred[3], double *const uf_out[3], void *stream);

/* Allocation-free stopping norms (the paper has no counterpart: this is a
 * library service).  For callers that cannot allocate device memory - their
 * device memory is owned by another allocator, or their time loop must not
 * call cudaMalloc/cudaFree, which can synchronise the whole device - and so
 * cannot create an mg_handle: computes the same per-field norms
 * ||D^-1 r||_2 as mg_residual_norms, with r = rhs - L(x) for the operator
 * that mg_apply applies, straight from the caller's arrays.
 *   grid: checked by the same rules as in mg_create.
 *   lambda [N][4], face_alpha[a] / face_k[a] (a < dim), rhs [N][2], x [N][2]:
 *     device pointers in the layouts described at the top of this file.
 *   out: device pointer to 2 doubles, receives (norm_T, norm_p).
 *   stream: cudaStream_t for the work; the call waits for it to finish
 *     before returning.
 * Allocates nothing: partial sums go to a static device array of 65536
 * entries (1 MiB on each device that runs it, kept until exit), so grids of
 * more than 65536 blocks of 32 x 8 cells (beyond 16,777,216 cells, e.g. 256^3
 * or 4096^2) are rejected with MG_ERR_INVALID_ARG.  The first call on each
 * device sets the scratch up (looks up its device address; with lazy module
 * loading, loads it and the kernels): make that first call before any stream
 * capture begins.  Each call rewrites every partial it later reads, so no
 * state carries over from the previous call, but all calls share the array:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller. */
MG_API mg_status mg_residual_norms_noalloc(const mg_grid *grid, const double *lambda,
                                           const double *const face_alpha[3], const double *const face_k[3],
                                           const double *rhs, const double *x, double *out, void *stream);

/* The current device's FP64 FMA issue rate in G FMA instructions per second
 * (no counterpart in the paper: the roofline denominator of the kernels bound
 * by the FP64 pipe).  A kernel of independent register-resident FMA chains
 * (4 blocks of 256 threads per SM, 8 chains per thread, no memory traffic)
 * runs once untimed and `repeats` (1..100) times timed with CUDA events on
 * `stream`; the fastest launch gives the rate.  Synchronous. */
MG_API mg_status mg_fp64_fma_rate(void *stream, int repeats, double *g_fma_per_s);

/* Copies `bytes` from page-locked host memory (mapped for the device, as
 * cudaHostAlloc / cudaMallocHost memory is) to device memory with a kernel on
 * `stream` (no counterpart in the paper: request transfers of the serving
 * loop).  The SMs load the source over the CPU-GPU link, so the copy does not
 * wait in the copy engines' queue behind a large transfer enqueued on another
 * stream; on a high-priority stream it runs beside that transfer.  Both
 * pointers 16-byte aligned; any size.  MG_ERR_INVALID_ARG (nothing launched)
 * for a source that is not page-locked host memory, a destination that is not
 * device memory of the current device, or misaligned pointers.  Asynchronous:
 * the source must stay valid and unchanged until the stream has run the copy. */
MG_API mg_status mg_copy_h2d_async(void *dst, const void *src, size_t bytes, void *stream);

/* ---------------------------------------------------------------------
 * Refined-patch (adaptive) grids.  The paper's production grids are coarsened
 * away from the bubble (Sec. 5.2, the rigid-wall collapse runs); here in its
 * two-level, block-structured form on 2D Cartesian grids: a uniform base grid
 * (spacing H, the grid's boundary conditions) and one box of base cells,
 * box[a][0] <= i < box[a][1] on axis a, refined 2:1 into a patch of spacing
 * H/2 ((2 * box width) cells per axis).  The unknowns are the patch's cells and
 * the base cells outside the box; each carries Eqs. 27-28 with its finite-volume
 * divergence:
 *   - between two cells of one level, and at the domain boundary: as on a
 *     uniform grid (walls: no flux; Dirichlet: the value half a cell away);
 *   - at the coarse-fine interface (a patch side inside the domain), seen from
 *     a patch cell: c_f (u~ - u_f) / (1.5 h), u~ = u_C + s (u_{C+t} - u_{C-t}) / 8
 *     the base field at the patch cell's tangential position (C the adjacent
 *     base cell, t along the interface, s = -1 for the lower, +1 for the upper
 *     of the two patch cells beside C; outside the domain the base cell's
 *     wall or Dirichlet ghost), 1.5 h being the distance between the two
 *     centres;
 *   - seen from the base cell C: the sum of its two patch faces' fluxes, with
 *     opposite sign (conservative).
 * Arrays: base [N_b][..] on the base grid's cells and faces, patch [N_f][..]
 * on the patch's (cells x-fastest, faces as for mg_set_coeffs), all device
 * pointers, pairs 16-byte aligned; a base cell under the box is ignored on
 * input and receives the mean of its four children on output.  FP64; the
 * calls wait for their work.
 * ------------------------------------------------------------------------- */
typedef struct mg_composite mg_composite;

/* grid: the base grid (dim 2, not axisymmetric; walls and Dirichlet sides);
 * box: base-cell range per axis, non-empty; opt: nu1, nu2, coarse_min and
 * coarse_solve of the cycles, and the precision: MG_FP64, or MG_MIXED, where
 * the FAC cycle's base correction runs its V-cycle in FP32 (with FP64 2x2
 * blocks at coefficient jumps, fp64_jump_ratio) while the composite
 * residuals, the patch sweeps and the update stay FP64 (NULL: defaults);
 * stream: cudaStream_t.  Allocates the base grid's hierarchy and the work
 * arrays. */
MG_API mg_status mg_composite_create(const mg_grid *grid, const int box[2][2], const mg_options *opt, void *stream,
                                     mg_composite **out);

/* Coefficients (Eqs. 29-32 and face 1/rho, k) of both levels, copied.  The base
 * hierarchy of the FAC cycle takes the base arrays outside the box and, under
 * it, the patch's coarsened: a covered cell's l1..l4 the mean of its children's,
 * each of its faces the mean of its two patch faces. */
MG_API mg_status mg_composite_set_coeffs(mg_composite *m, const double *lam_b, const double *const fa_b[3],
                                         const double *const fk_b[3], const double *lam_f,
                                         const double *const fa_f[3], const double *const fk_f[3]);

/* y = L(x) on the composite grid (with the grid's Dirichlet values); yb of the
 * covered base cells is 0. */
MG_API mg_status mg_composite_apply(mg_composite *m, const double *xb, const double *xf, double *yb, double *yf);

/* The paper's defect-correction loop (Sec. 3, after Eq. 34) for L(x) = b,
 * `cycles` steps, each correction one FAC cycle: nu1 red-black block
 * Gauss-Seidel sweeps on the patch rows (interface values of the base
 * correction zero), the patch residual averaged onto the covered base cells
 * and the valid base cells' residual corrected for the patch's interface
 * fluxes, one V-cycle of the base hierarchy from zero, its result prolonged
 * onto the patch (cell-centred bilinear) and added, nu2 sweeps on the patch
 * rows with the base correction's interface values; then x += the correction
 * on the valid cells.  norms (nullable, host, 4 * (cycles + 1)): before each
 * step and after the last, the L2 norms of the T and p residuals over the
 * valid base cells, then over the patch. */
MG_API mg_status mg_composite_solve(mg_composite *m, const double *bb, const double *bf, double *xb, double *xf,
                                    int cycles, double *norms);

/* Measures and applies the kernel choices of the base grid's hierarchy, as
 * mg_autotune does for a handle (every choice runs the same arithmetic, so
 * later solves give the same result bit for bit).  Needs coefficients.
 * vcycle_ms (nullable, host): the chosen V-cycle's time.  Waits for its
 * work. */
MG_API mg_status mg_composite_autotune(mg_composite *m, int reps, double *vcycle_ms);

MG_API mg_status mg_composite_destroy(mg_composite *m);

/* Moves all later work of the handle to another stream (cudaStream_t on the
 * handle's device).  The new stream waits, on the device, for the work that
 * the handle's last mg_set_coeffs or mg_solve_async left running (the other
 * calls finish theirs before returning); the call does not block the host and
 * does not wait for later work of other handles on the old stream. */
MG_API mg_status mg_set_stream(mg_handle *h, void *stream);

/* Makes `device` the CUDA device this thread's later mg_create calls use
 * (the library's own runtime keeps a current device per thread). */
MG_API mg_status mg_set_device(int device);

/* Number of multigrid levels and the finest-to-coarsest sizes (n_out: levels x 3 ints, may be NULL). */
MG_API mg_status mg_levels(const mg_handle *h, int *levels, int *n_out);

MG_API mg_status mg_destroy(mg_handle *h);

/* Message of the calling thread's last failure ("" if none). */
MG_API const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* COUPLEDMG_H */
