/*
 * tmg -- time multigrid for DG-in-time discretisations on one GB300 (sm_103a).
 *
 * C ABI of the GPU library libtmg.so.  Plain pointers and sizes only; every
 * array argument of tmg_solve / tmg_cycle / tmg_residual is a DEVICE pointer
 * on the plan's CUDA stream unless its name ends in _host.
 *
 * The problem (Gander & Neumueller, arXiv:1409.5254, Section 2, eq.
 * chap4_generalLinearSystemODE, generalised to u' + lambda u = f):
 *
 *   (K + z Mhat) u_n = f_n + N u_{n-1},  n = 1..N,  z = lambda * tau,
 *
 * with the degree-p_t shifted Legendre basis psi_k(s) = P_k(2s - 1) on each
 * interval, K the upwind DG stiffness block, Mhat the reference mass matrix,
 * N = a b^T (a_k = psi_k(0) = (-1)^k, b_l = psi_l(1) = 1) and u_0 := the initial
 * value.  Array layout: interval-major [N][p_t + 1] float64, i.e. element
 * (n, k) (0-based interval n, Legendre coefficient k) at offset n*(p_t+1)+k.
 * The right-hand side f is the assembled load vector f_n[k] = int f psi_k^n dt
 * (Section 2, definition of the right-hand sides); the initial value enters as
 * a*u0 in the first interval inside the library (f is never modified).
 *
 * The solver is the paper's multigrid in time (Section 3): damped block Jacobi
 * smoothing (eq. chap4_ODESmoother) with the damping omega* of Lemma
 * chap4_lemma7 per level, restriction R = [R1 R2] and prolongation P = R^T
 * (eqs. chap4_restrictionTime, chap4_prolongationTime), V- or W-cycles on
 * factor-2 coarsened meshes (eq. chap4_errorTwoGridCycle), and an exact
 * coarsest solve by a parallel prefix scan over affine interval maps.  Each
 * cycle is a correction step: r = F - L u in FP64, one cycle on L c = r in
 * the cycle precision (FP64, or FP32 for TMG_MIXED), u += c in FP64.  The
 * mixed form by default keeps r between cycles as a float pair updated by
 * r -= L c (no FP64 operation) and recomputes it from u only at the start of
 * a solve and to confirm convergence.  The stopping test is
 * ||F - L u||_2 <= tol * ||F||_2 with F - L u evaluated from u in FP64.
 *
 * Errors: every function returns a tmg_status; nothing aborts or exits.  A
 * failed CUDA call returns TMG_ECUDA (the CUDA error is kept, see
 * tmg_last_cuda_error).  Plans are not thread-safe; use one plan per host
 * thread or serialise calls.
 */
#ifndef TMG_H
#define TMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tmg_plan tmg_plan;

typedef enum {
    TMG_OK = 0,
    TMG_EINVAL = 1,     /* bad argument (see tmg_setup for the rules) */
    TMG_ENOMEM = 2,     /* device or host allocation failed */
    TMG_ECUDA = 3,      /* a CUDA runtime call failed */
    TMG_ENOTCONV = 4,   /* max_cycles reached before tol; u holds the last iterate */
    TMG_ENUMERIC = 5,   /* a residual norm was NaN or Inf */
    TMG_ETIMEOUT = 6,   /* a bounded device-side wait ran out */
    TMG_EUNSUPPORTED = 7 /* valid request this build does not implement */
} tmg_status;

enum { TMG_FP64 = 0, TMG_MIXED = 1 };

typedef struct {
    double tol;         /* relative residual target ||F-Lu||/||F|| (default 1e-10) */
    int max_cycles;     /* cycle limit (default 100) */
    int nu1, nu2;       /* pre/post smoothing sweeps (default 1, 1); 0..8 */
    int gamma;          /* 1 = V-cycle, 2 = W-cycle (default 1) */
    int precision;      /* TMG_FP64 or TMG_MIXED (default TMG_MIXED) */
    int64_t n_min;      /* coarsen while N_l is even and N_l > n_min (default 64) */
    int use_graph;      /* 1: whole solve as one CUDA graph launch (default 1) */
    int initial_guess;  /* 1: tmg_solve starts from the u passed in (default 0: u = 0) */
    int64_t tail_cap;   /* most intervals the on-chip coarse solver takes (0: default, 64 for
                           V-cycles, 8192 for W-cycles, 2048 for W-cycles of batches; at most
                           8192); smaller values move more levels to the streaming kernels */
    int use_pdl;        /* 1: programmatic dependent launch between the kernels of a cycle,
                           hiding each launch behind its predecessor's tail (default 1) */
    int update_residual; /* TMG_MIXED: 1 = keep the level-0 residual as a float pair (about
                           39 bits stored) updated by r -= L c after each cycle, recomputed from u in
                           FP64 only at the start and to confirm convergence (default 1);
                           0 = recompute it from u in FP64 every cycle */
    int fuse_levels;    /* 1: the streaming levels l >= 1 run two per kernel (levels l and
                           l+1 on the way down and up, level l+1 never stored; the way up
                           recomputes level l+1's right-hand side); 0: one level per
                           kernel; -1 (default): fuse when the cycle precision is FP32 */
    int schedule;       /* batches: how each (p_t, length) group runs.  TMG_SCHED_AUTO
                           (default): time both forms at setup on a synthetic problem and
                           keep the faster; TMG_SCHED_GRID: level kernels over all instances
                           of the group (graph loop); TMG_SCHED_CTA: one CTA per instance with
                           the whole hierarchy in shared memory and all cycles in one launch
                           (groups too large for one CTA fall back to the grid form) */
    int check_fp64;     /* 1: after each solve, also solve the system exactly in FP64 (the
                           parallel scan of tmg_solve_direct; for batches one warp per
                           instance) and record max|u - u_exact| / max|u_exact|, reported by
                           tmg_stats / tmg_stats_batched as err_vs_fp64 (default 0: not
                           computed, reported as NAN).  Costs one exact solve per solve and,
                           for a single problem, an N (p_t+1) double buffer owned by the plan */
} tmg_opts;

enum { TMG_SCHED_AUTO = 0, TMG_SCHED_GRID = 1, TMG_SCHED_CTA = 2 };

/* Fill *opts with the defaults listed above. */
void tmg_opts_default(tmg_opts *opts);

/*
 * Build a plan for one problem: degree p_t in 0..5, 10 or 20 (the degrees of
 * the paper's scaling tables; at 10 and 20 the coarsest level is always solved
 * by the grid-wide scan and the mixed form recomputes the level-0 residual
 * from u in every cycle, as with update_residual = 0), step tau > 0,
 * lambda >= 0 (finite), N >= 1 intervals.  levels <= 0 picks the hierarchy
 * from opts->n_min; levels >= 1 caps the number of levels.  omega <= 0 uses
 * omega*(alpha(lambda tau_l)) per level (Lemma chap4_lemma7); 0 < omega < 2
 * uses that damping on every level (omega in (1,2) converges but not
 * uniformly, remark after Theorem chap4_theorem3).  stream is a cudaStream_t
 * (NULL = legacy default stream).  All setup arithmetic is FP64 on the host
 * (block inverses, alpha, omega*, transfer matrices); the library allocates
 * and owns every workspace.  The levels below the first one that fits on one
 * SM's shared memory run in a single-CTA coarse solver; when even the
 * coarsest level is too large for that, it is solved exactly by a grid-wide
 * scan (see tmg_solve_direct).  W-cycles (gamma = 2) visit every level below
 * level 0 twice per visit of its parent, the second visit starting from the
 * first one's result (one launch per level and visit on the streaming levels,
 * so their cost in launches doubles per level: keep the streaming part short
 * with the default tail_cap).  Returns TMG_EINVAL for bad arguments (p_t
 * outside 0..20 among them), TMG_EUNSUPPORTED for the other degrees up to 20,
 * TMG_ENOMEM / TMG_ECUDA on allocation failure.
 */
tmg_status tmg_setup(tmg_plan **plan, int p_t, double tau, double lambda, int64_t N, int levels,
                     double omega, const tmg_opts *opts, void *stream);

/*
 * Solve L u = F.  f: device [N][p_t+1] load vector (read only); u0: initial
 * value; u: device [N][p_t+1] output (input too when opts->initial_guess).
 * f and u must be 16-byte aligned and must not overlap.  Returns TMG_OK when
 * the FP64 relative residual reached tol, TMG_ENOTCONV after max_cycles.
 * Synchronises the plan's stream before returning.
 */
tmg_status tmg_solve(tmg_plan *plan, const double *f, double u0, double *u);

/*
 * Same solve with HOST arrays: copies f_host to the device, solves, copies u
 * back (all on the plan's stream, inside the call).  Pinned host memory gives
 * full copy bandwidth; pageable memory works too.
 */
tmg_status tmg_solve_host(tmg_plan *plan, const double *f_host, double u0, double *u_host);

/*
 * Exact FP64 solve of L u = F without multigrid, by a parallel prefix scan.
 * N = a b^T has rank one, so block forward substitution (the plain solution of
 * eq. chap4_generalLinearSystemODE) is the scalar recurrence
 * e_n = alpha e_{n-1} + c^T F_n for e_n = b^T u_n, then u_n = A^{-1} F_n +
 * g e_{n-1}; affine maps compose associatively, and three passes (tile maps,
 * tile prefixes, replay) evaluate it in parallel reading F once more than the
 * minimum.  Not the paper's method: the reference the multigrid solve is
 * measured against.  Arguments as for tmg_solve; synchronises the stream.
 */
tmg_status tmg_solve_direct(tmg_plan *plan, const double *f, double u0, double *u);

/*
 * Gradients of a loss J(u) at the solution u of L u = F, through the adjoint
 * system L^T mu = g with g = dJ/du (device [N][p_t+1]).  L^T has diagonal
 * blocks A^T and super-diagonal blocks -N^T = -b a^T (the transpose of eq.
 * chap4_generalLinearSystemODE), i.e. it couples each interval to the NEXT
 * one; read in reversed time it has the same block lower-bidiagonal form, so
 * the library solves it with the same multigrid cycle on reversed arrays (the
 * transfer operators keep R = P^T; the Galerkin identity transposes).  The
 * plan's tolerance applies relative to ||g||.  Outputs: dJdf = mu (device
 * [N][p_t+1]); *dJdu0 = a^T mu_1 (u0 enters F_1 as a*u0); *dJdlambda =
 * -tau sum_n mu_n^T Mhat u_n (L depends on lambda through lambda*tau*Mhat);
 * dJdu0 and dJdlambda are device doubles.  u must be the forward solution.
 * The first call allocates a 2 N (p_t+1) double buffer owned by the plan.
 */
tmg_status tmg_adjoint(tmg_plan *plan, const double *g, const double *u, double *dJdf, double *dJdu0,
                       double *dJdlambda);

/*
 * Apply exactly one correction cycle to u in place (no convergence test):
 * u <- u + C (F - L u) with C one V/W-cycle in the plan's precision.
 */
tmg_status tmg_cycle(tmg_plan *plan, const double *f, double u0, double *u);

/*
 * Error of a result u against the exact FP64 solution of the same system:
 * *err = max|u - u_exact| / max|u_exact| (host double), with u_exact the
 * FP64 parallel-scan solve of tmg_solve_direct (block forward substitution of
 * eq. chap4_generalLinearSystemODE written as a scan), held in an
 * N (p_t+1) double buffer the plan allocates on first use.  tmg_stats reports
 * the value afterwards as err_vs_fp64.  f, u device arrays as for tmg_solve;
 * synchronises the stream.
 */
tmg_status tmg_error_vs_fp64(tmg_plan *plan, const double *f, double u0, const double *u, double *err);

/*
 * One correction cycle split at the plan's coarsest level, for callers that
 * solve that level themselves -- the time-slab partition of one long horizon
 * over several GPUs, where every slab's coarsest-level right-hand sides are
 * gathered and the coarse part of the cycle (eq. chap4_errorTwoGridCycle
 * below that level) runs on the gathered problem.  tmg_cycle_down evaluates
 * r = F - L u (FP64) and runs the way down of one V-cycle on L c = r:
 * pre-smoothing, residual and restriction on every level above the coarsest,
 * whose right-hand side it writes to fc (device, N_c (p_t+1) doubles, N_c the
 * coarsest level's intervals, tmg_plan_info).  tmg_cycle_up takes that
 * level's correction uc (device, same size), runs the way up (prolongation,
 * post-smoothing on every level) and updates u += c; u must be the array
 * passed to the tmg_cycle_down call it completes.  Together with uc = the
 * exact or multigrid correction of the coarsest level they apply the same
 * cycle as tmg_cycle.  The plan must run V-cycles, have at least two levels,
 * no on-chip solver above its coarsest level (opts->tail_cap = 1), and no
 * updated level-0 residual (TMG_FP64, or update_residual = 0): else
 * TMG_EUNSUPPORTED.  Both synchronise the stream.
 */
tmg_status tmg_cycle_down(tmg_plan *plan, const double *f, double u0, double *u, double *fc);
tmg_status tmg_cycle_up(tmg_plan *plan, const double *uc, double *u);

/* r = F - L u (FP64, device arrays [N][p_t+1]); F is f with a*u0 folded in. */
tmg_status tmg_residual(tmg_plan *plan, const double *f, double u0, const double *u, double *r);

/*
 * Statistics of the last tmg_solve: number of cycles applied, final relative
 * residual, the error against the exact FP64 solution (*err_vs_fp64 =
 * max|u - u_exact| / max|u_exact|, u_exact the FP64 parallel-scan solve of the
 * same system, as tmg_solve_direct; NAN unless the plan was built with
 * opts->check_fp64), and up to hist_len entries of the residual history
 * (hist[k] = ||F - L u_k|| / ||F||, k = 0..cycles).  Any pointer may be NULL.
 */
tmg_status tmg_stats(const tmg_plan *plan, int *cycles, double *rel_res, double *err_vs_fp64, double *hist,
                     int hist_len);

/*
 * The hierarchy tmg_setup builds for these arguments, computed on the host
 * without touching the GPU (the same code tmg_setup runs): the number of
 * levels (coarsening while a level has an even number of intervals, more
 * than opts->n_min of them, and the level cap allows, Section 3's nested
 * meshes); the first level handed to the single-CTA coarse solver; its
 * number of intervals; and *scan_coarsest = 1 when no level fits that solver
 * (or p_t = 10, 20) and the coarsest level is solved by the grid-wide scan
 * instead.  Output pointers are host pointers and may be NULL.  Same
 * argument checks and status codes as tmg_setup.
 */
tmg_status tmg_plan_shape(int p_t, double tau, double lambda, int64_t N, int levels, double omega,
                          const tmg_opts *opts, int *num_levels, int *tail_level, int64_t *tail_intervals,
                          int *scan_coarsest);

/*
 * The FP64 set-up arithmetic of one level at step z = lambda*tau_l, on the
 * host (what tmg_setup uploads per level): A = K + z Mhat (Section 2, the
 * local matrices in the shifted Legendre basis), its inverse, g = A^{-1} a,
 * c = A^{-T} b (so that c^T f = b^T A^{-1} f), alpha = b^T A^{-1} a (Lemma
 * chap4_theorem2), and the damping: omega_user if 0 < omega_user < 2, else
 * omega* of Lemma chap4_lemma7.  A and Ainv are row-major (p_t+1)^2 host
 * arrays, g and c (p_t+1); any output may be NULL.  p_t and z >= 0 as for
 * tmg_setup (TMG_EINVAL / TMG_EUNSUPPORTED likewise).
 */
tmg_status tmg_level_constants(int p_t, double z, double omega_user, double *A, double *Ainv, double *g,
                               double *c, double *alpha, double *omega);

/*
 * The prolongation matrices P1 = R1^T and P2 = R2^T of Section 4.2 (eqs.
 * chap4_restrictionTime / chap4_prolongationTime): column k holds the fine
 * Legendre coefficients of coarse basis function k on the first (second)
 * half of the coarse interval.  Row-major (p_t+1)^2 host arrays; host only.
 */
tmg_status tmg_transfer_matrices(int p_t, double *P1, double *P2);

/* Level count and the first level handled by the on-chip coarse solver. */
tmg_status tmg_plan_info(const tmg_plan *plan, int *num_levels, int *tail_level, int64_t *tail_intervals,
                         double *omega_per_level, int omega_len);

/*
 * Kernels one correction cycle launches (every kernel of the solve's graph
 * body, including those that return at once), as counted when the cycle was
 * last enqueued (a solve, tmg_cycle or tmg_profile_cycle); 0 before that.
 * A solve of k cycles runs the body k + 1 times (the last one confirms the
 * residual from u).
 */
tmg_status tmg_plan_launches(const tmg_plan *plan, int *per_cycle);

/*
 * Measurement helper: apply reps correction cycles to u (as tmg_cycle) with a
 * CUDA event recorded on the plan's stream around every kernel, and return the
 * mean milliseconds per cycle in ms[0..5]: level-0 down kernel (or the level-0
 * residual when the whole correction runs on chip), all streaming down kernels
 * of levels >= 1, the on-chip coarse solver, all streaming up kernels, the
 * level-0 up kernel (or update), and the whole cycle.  n_ms >= 6.
 */
tmg_status tmg_profile_cycle(tmg_plan *plan, const double *f, double u0, double *u, int reps, double *ms,
                             int n_ms);

/*
 * Copy one of the plan's internal level vectors to host memory (inspection
 * and testing; synchronises the stream).  which: 0 = right-hand side f_l,
 * 1 = correction u_l of level l (levels 0..tail level), 2 = the level-0
 * residual r (level ignored), 3 = the low float parts of that residual when
 * the plan keeps it as a float pair (TMG_MIXED with update_residual; the
 * residual is then r + low, else TMG_EINVAL).  The vector holds N_l*(p_t+1)
 * values of the cycle precision (8-byte double for TMG_FP64, 4-byte float for
 * TMG_MIXED; always float for 3); bytes must be at least that size.
 */
tmg_status tmg_inspect(const tmg_plan *plan, int which, int level, void *host_dst, size_t bytes);

/*
 * Residual r = F - L u (FP64, written to r) and its norm ||r||_2 (written to
 * the single device double *norm), with no plan and no device allocation --
 * for callers that may not allocate device memory where they need this check
 * (real-time loops that cannot take the device synchronisation an allocation
 * may cause, applications whose device memory all belongs to their own
 * pool).  The paper has no counterpart;
 * it is the level-0 residual kernel with its block partial sums kept in a
 * fixed file-scope device array instead of a plan workspace.
 *
 * p_t (0..5), tau, lambda, N, f, u0, u as for tmg_setup/tmg_solve; f, u, r device
 * [N][p_t+1] float64, 16-byte aligned; norm an 8-byte aligned device double.
 * N may not exceed 2^21 intervals (the scratch array holds 1024 block partial
 * sums of 2048 intervals each): larger N returns TMG_EUNSUPPORTED before any
 * GPU work.  The first call on a device looks up the scratch array's device
 * address with that device current; make that first call before any stream
 * capture.  Every call on a device shares the array and leaves its contents
 * behind; calls whose kernels may overlap on the GPU (unordered streams) race
 * on it and must be serialised by the caller.  Asynchronous on stream
 * (a cudaStream_t; NULL = legacy default stream).
 */
tmg_status tmg_residual_norm_noalloc(int p_t, double tau, double lambda, int64_t N, const double *f, double u0,
                                     const double *u, double *r, double *norm, void *stream);

/* ------------------------------------------------------------ batches -- */

typedef struct tmg_batch tmg_batch;

/*
 * Plan for n_inst (1 <= n_inst <= 2^31 - 1) independent problems
 * u' + lambda_i u = f_i, u(0) = u0_i, instance i with degree p_t[i] in
 * {0..5, 10, 20}, step tau[i] > 0, lambda[i] >= 0 and N[i] >= 1 intervals
 * (host arrays of length n_inst).  Packed layout of every
 * [instance][interval][coefficient] array: instance i starts at value offset
 * off_i = sum_{j<i} N[j] (p_t[j] + 1).  omega and opts as for tmg_setup;
 * levels coarsen while even and longer than nmin = min(opts->n_min, 64)
 * intervals, the coarsest level solved exactly.  Internally the instances are
 * grouped: an instance whose own hierarchy coarsens at least once down to at
 * most nmin intervals joins the group of its degree and depth and is solved on
 * its own intervals with its own hierarchy (the level kernels tile only real
 * intervals); any other instance (at most 64 intervals, or an odd coarsest
 * level longer than nmin) is padded at its end to a power-of-two length (the
 * system is causal, so this leaves its solution unchanged).  Every level
 * kernel covers all instances of a group still iterating at once.
 * W-cycles (gamma = 2) visit every level below level 0 twice per visit of
 * its parent: in the grid form the streaming levels down to the first one of
 * at most tail_cap (default 2048) intervals are launched once per visit, and the levels from
 * there on run in one CTA per instance, whose shared-memory recursion makes
 * its own visits; the CTA form runs the whole W recursion on chip.  Degrees
 * 10 and 20 run V-cycles in the grid form, the level-0 residual recomputed
 * from u in every cycle.  Per-instance FP64 constants are computed on the
 * host.  Returns as tmg_setup.
 */
tmg_status tmg_setup_batched(tmg_batch **batch, int64_t n_inst, const int *p_t, const double *tau,
                             const double *lambda, const int64_t *N, double omega, const tmg_opts *opts,
                             void *stream);

/*
 * Solve every instance: f, u device packed arrays (16-byte aligned), u0
 * device [n_inst].  Each instance stops on its own test ||F_i - L_i u_i|| <=
 * tol ||F_i|| (its lanes are frozen afterwards); TMG_ENOTCONV if any instance
 * reached max_cycles.  Synchronises the stream.
 */
tmg_status tmg_solve_batched(tmg_batch *batch, const double *f, const double *u0, double *u);

/*
 * Gradients of a loss through every instance's adjoint (see tmg_adjoint):
 * g = dJ/du and u (the forward solutions) packed device arrays; outputs
 * dJdf (packed), dJdu0[n_inst] and dJdlambda[n_inst] on the device.
 */
tmg_status tmg_adjoint_batched(tmg_batch *batch, const double *g, const double *u, double *dJdf, double *dJdu0,
                               double *dJdlambda);

/* Per-instance cycles, final relative residuals and errors against the exact
 * FP64 solution (max|u_i - u_exact,i| / max|u_exact,i|, NAN unless the batch
 * was built with opts->check_fp64) of the last batched solve (host arrays of
 * length n_inst, may be NULL); *max_cycles_used = the most. */
tmg_status tmg_stats_batched(const tmg_batch *batch, int *cycles, double *rel_res, double *err_vs_fp64,
                             int *max_cycles_used);

/*
 * Errors of the batched results u against every instance's exact FP64
 * solution, err_host[i] = max|u_i - u_exact,i| / max|u_exact,i| (host array of
 * n_inst): one warp per instance composes the affine maps of contiguous chunks
 * of the recurrence e_n = alpha e_{n-1} + c^T F_n, scans them across the warp
 * and replays each chunk (exact block forward substitution, FP64).  f, u0, u
 * device arrays as for tmg_solve_batched; tmg_stats_batched reports the values
 * afterwards.  Synchronises the stream.
 */
tmg_status tmg_error_vs_fp64_batched(tmg_batch *batch, const double *f, const double *u0, const double *u,
                                     double *err_host);

/* Number of groups and the number of values the level kernels cover (the real
 * values of variable-length groups, the padded slots of power-of-two ones). */
tmg_status tmg_batch_info(const tmg_batch *batch, int *n_groups, int64_t *padded_values);

/*
 * The autotuner's whole-batch check (schedule TMG_SCHED_AUTO): per-group
 * times are taken one group at a time, but a solve runs all groups at once,
 * so when some group chose the CTA form the setup also times one solve of the
 * whole synthetic batch with the per-group choices (*ms_tuned) and with every
 * group on the grid form (*ms_grid), and keeps the faster.  Both are NAN when
 * the check did not run (one group, no CTA choice, or another schedule).
 */
tmg_status tmg_batch_tune_info(const tmg_batch *batch, double *ms_tuned, double *ms_grid);

/*
 * Group g (0 <= g < n_groups): degree, padded length, instances, the schedule
 * it runs (TMG_SCHED_GRID or TMG_SCHED_CTA), and the milliseconds the setup
 * autotuner measured for one synthetic solve in each form (NAN where a form
 * was not timed).  Any output pointer may be NULL.
 */
tmg_status tmg_batch_group_info(const tmg_batch *batch, int g, int *p_t, int64_t *padded_length,
                                int64_t *n_instances, int *schedule, double *ms_grid, double *ms_cta);

void tmg_destroy_batched(tmg_batch *batch);

/* ----------------------------------------------- space-time heat -- */

typedef struct tmg_heat tmg_heat;

/*
 * The paper's outlook (Section 7): the heat equation u_t - Delta u = f on the
 * unit square, zero Dirichlet boundary values, the 5-point finite-difference
 * Laplacian A_h on an n x n interior grid (h = 1/(n+1), n = 2^k - 1), and the
 * DG-in-time discretisation of Section 2 of degree p_t (0..5) with N = 2^j
 * steps of size tau.  The system is block lower-bidiagonal (eq.
 * chap4_generalLinearSystemODE with lambda replaced by A_h): diagonal blocks
 * G = K (x) I + tau Mhat (x) A_h, sub-diagonal blocks -(a b^T) (x) I.  Arrays
 * are device FP64, [N][p_t+1][n][n] (interval, Legendre coefficient, row,
 * column); f is the load vector, u0 the initial field [n][n].
 *
 * The solver is the time multigrid of Section 3 with the damped block Jacobi
 * smoother of eq. chap4_ODESmoother (omega = 1/2, the uniform damping that
 * bounds the smoothing factor of every spatial mode), in which each block
 * inverse is replaced by one multigrid V(1,1)-cycle in space (damped
 * point-block Jacobi omega = 4/5, full weighting, bilinear prolongation,
 * down to one grid point); time coarsens by two to one interval, solved by
 * nu_c (1..16) spatial V-cycles.  opts: tol, max_cycles, nu1, nu2 (V-cycles
 * only, gamma = 1), use_graph (each cycle replayed from a CUDA graph captured
 * at its first use for the given arrays), precision: TMG_FP64 (every step in
 * FP64, the textbook iterates) or TMG_MIXED (the residual of the FP64 iterate
 * formed in FP64, one cycle in FP32 from a zero correction c, u += c in FP64;
 * iterative refinement to the same FP64 tolerance).  The convergence test
 * always uses the FP64 residual.  n <= 2^14 - 1, N <= 2^40.  Returns
 * TMG_EINVAL for other sizes or options, TMG_ENOMEM when the workspace
 * (about 7 N (p_t+1) n^2 values of the cycle precision) does not fit.
 */
tmg_status tmg_heat_setup(tmg_heat **plan, int p_t, double tau, int n, int64_t N, const tmg_opts *opts, int nu_c,
                          void *stream);

/* Cycles from u = 0 until ||F - L u|| <= tol ||F|| (F: f with a (x) u0 in the
 * first interval); TMG_ENOTCONV after max_cycles.  Synchronises the stream. */
tmg_status tmg_heat_solve(tmg_heat *plan, const double *f, const double *u0, double *u);

/* Exactly one cycle applied to u in place. */
tmg_status tmg_heat_cycle(tmg_heat *plan, const double *f, const double *u0, double *u);

/* r = F - L u (device arrays as above). */
tmg_status tmg_heat_residual(tmg_heat *plan, const double *f, const double *u0, const double *u, double *r);

/* Cycles and relative residual of the last tmg_heat_solve, and up to hist_len
 * entries of its residual history; any pointer may be NULL. */
tmg_status tmg_heat_stats(const tmg_heat *plan, int *cycles, double *rel_res, double *hist, int hist_len);

/* Diagnostics: CUDA-event times on the plan's stream (ms per launch, mean of
 * reps) of the level-0 kernels after one cycle from u: ms[0] the time
 * residual in the cycle precision, ms[1] the fused pre-smoothing, residual
 * and restriction of spatial level 0, ms[2] the fused prolongation and
 * post-smoothing of spatial level 0 accumulating into a work array, ms[3]
 * the mixed form's float-pair residual update (u += c, r -= L c) or the FP64
 * form's FP64 residual, ms[4] one whole cycle.  n_ms >= 5.  u is left
 * arbitrary (solve again afterwards). */
tmg_status tmg_heat_profile(tmg_heat *plan, const double *f, const double *u0, double *u, int reps, double *ms,
                            int n_ms);

/* Time and spatial levels of the hierarchy, kernels (and memsets) one cycle
 * issues after its first use (0 before), workspace bytes; any pointer may be
 * NULL. */
tmg_status tmg_heat_info(const tmg_heat *plan, int *time_levels, int *space_levels, int *launches_per_cycle,
                         size_t *workspace_bytes);

void tmg_heat_destroy(tmg_heat *plan);

/* Release the plan and every resource it owns.  NULL is ignored. */
void tmg_destroy(tmg_plan *plan);

/* Static text for a status code. */
const char *tmg_strerror(tmg_status status);

/* Last CUDA error code seen by the library in this process (0 if none). */
int tmg_last_cuda_error(void);

/* Debug build only (the library compiled with -DTMG_BOUNDS): the number of
 * out-of-range indices its kernels met since the last call, and the first
 * (site << 40 | low 40 bits of the index; sites are listed in
 * csrc/tmg_bounds.h), both cleared.  Each such access was skipped (a load
 * gave 0).  Returns TMG_EUNSUPPORTED from the normal build. */
tmg_status tmg_debug_bounds(unsigned *violations, unsigned long long *first);

#ifdef __cplusplus
}
#endif

#endif /* TMG_H */
