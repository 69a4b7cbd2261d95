/*
 * ps.h -- C ABI of the GB300 parareal + splitting solver.
 *
 * Method: Arraras, Gaspar, Jimenez-Ciga, Portero, "Space-time parallel
 * iterative solvers for the integration of parabolic problems",
 * arXiv 2502.08370.  The library integrates
 *     u_t = div(a grad u) - c u + f   on the unit square / cube,
 *     u = 0 on the boundary                         (Sec. 2.1, eq. cont_problem)
 * discretised by second-order finite differences on a uniform grid of
 * interior nodes (Sec. 2.2, eq. semidisc_prob; Sec. 5), split either by
 * dimension (x/y/z) or by a partition of unity over overlapping boxes
 * (Sec. 2.1), advanced by fractional implicit Euler steps (Sec. 2.2,
 * eq. FIE_method) used as both propagators of the parareal iteration
 * (Sec. 3, Parareal/FIE-FIE of Sec. 4).
 *
 * Conventions for every entry point:
 *  - Return value: PS_OK (0) or a PS_ERR_* code; ps_last_error() gives a
 *    message for the calling thread's last failure.  No entry point aborts.
 *  - Arrays are dense, x fastest: a state has nx*ny*nz doubles (interior
 *    nodes, boundary values are the implicit zero Dirichlet data); a nodal
 *    coefficient has (nx+2)*(ny+2)*(nz+2) doubles (boundary included).
 *    nz = 1 in 2-D.
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library reads or writes them on the given stream and never frees them.
 *    Pointers named *_host are host pointers (pinned or pageable).
 *  - `stream` is a cudaStream_t passed as uintptr_t (0 = legacy default).
 *    Work is enqueued on it; functions that return host data synchronise it.
 *  - Handles are opaque, owned by the library, freed by the matching
 *    *_destroy.  A problem keeps pointers to its splittings, a splitting to
 *    its operator, an operator to its grid: destroy in reverse order.
 *  - The library allocates its own device workspaces with cudaMalloc at
 *    handle creation (PS_ERR_OOM when that fails) and frees them on destroy.
 */
#ifndef PS_H
#define PS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PS_OK 0
#define PS_ERR_INVALID 1        /* bad argument or state */
#define PS_ERR_CUDA 2           /* a CUDA runtime call failed (message has the CUDA error) */
#define PS_ERR_OOM 3            /* device allocation failed */
#define PS_ERR_NONFINITE 4      /* a NaN/Inf appeared in the parareal correction */
#define PS_ERR_DEVICE_TIMEOUT 5 /* a device-side wait ran out of its time limit (0.5 s) */
#define PS_ERR_UNSUPPORTED 6    /* combination not implemented (e.g. 3-D DD splitting) */

#define PS_SPLIT_DIM 0 /* dimensional splitting, M = d substeps x, y(, z) (Sec. 2.1) */
#define PS_SPLIT_DD 1  /* domain-decomposition splitting, 2-D, M = #colours (Sec. 2.1) */

#define PS_PREC_FP64 0  /* every solve in FP64 */
#define PS_PREC_MIXED 1 /* fine-propagator line solves in FP32; the coarse propagator (FP64
                           unless PS_COARSE_DELTA32), the parareal correction, the increments
                           and the test in FP64 */

/* Coarse propagator arithmetic (ps_params.coarse).  G is affine (Sec. 2.2, eq. FIE_method:
 * G(u) = B u + c with c from the source), so the bracket G(U_n^k) - G(U_n^{k-1}) of the
 * parareal correction equals B (U_n^k - U_n^{k-1}).  PS_COARSE_DELTA32 evaluates it in that
 * form with FP32 line solves on the FP32-rounded increment: the rounding is relative to the
 * increment, not to U, so the FP64 increment test still reaches small tolerances.  The
 * correction U_{n+1}^k = F(U_n^{k-1}) + B d_n, the increments and the test stay FP64; the
 * initial coarse sweep U_{n+1}^0 = G(U_n^0) runs with FP32 line solves on the state.
 * Finite termination stays bitwise (d_n = 0 gives B d_n = 0).  Dimensional splitting only;
 * not in batches or adjoints.  ps_run_coarse_sequential keeps the FP64 coarse steps. */
#define PS_COARSE_FP64 0    /* G in FP64, correction written as F + (G_new - G_old) (Sec. 3) */
#define PS_COARSE_DELTA32 1 /* G's linear part in FP32 on the increment, see above */

/* Fine propagator (ps_params.fine_method).  PS_FINE_DR takes s Douglas-Rachford steps
 * (Sec. 2.2, eq. DR_method) per slice: Parareal/FIE-DR of Sec. 4.2, G staying FIE.
 * PS_PREC_FP64 only, with the dimensional or the DD splitting; not in batches or adjoints. */
#define PS_FINE_FIE 0 /* fractional implicit Euler (eq. FIE_method) */
#define PS_FINE_DR 1  /* Douglas-Rachford (eq. DR_method) */

/* Line-solve schedule (ps_params.schedule) of the coarse propagator's x-substep (the sweep
 * over contiguous rows on one slice; dimensional splitting).  Every other line solve runs the
 * Thomas/LDL^T recurrences one thread per line (fine tiles, coarse y/z sweeps staged or
 * streamed, PS_COARSE_SWEEP_*).  The schedules compute the same solution in different orders:
 * the coarse values change at rounding level (FP32 for the increment form, FP64 otherwise), the
 * parareal fixed point does not.  PCR is built for the FP32 increment form (rows of at most 256
 * nodes; PS_ERR_UNSUPPORTED otherwise). */
#define PS_SCHED_AUTO 0   /* FP32 increment form: the hybrid; FP64 coarse: Thomas; unless ps_autotune
                             picked another */
#define PS_SCHED_THOMAS 1 /* Thomas/LDL^T recurrences, one thread per row */
#define PS_SCHED_PCR 2    /* parallel cyclic reduction, one warp per row (log2 L shuffle/register steps) */
#define PS_SCHED_HYBRID 3 /* one warp per row: lane segments run sequentially, a log-depth shuffle scan
                             joins them (segmented scans of the two first-order recurrences) */

/* Schedules of the coarse propagator's line solves (ps_params.coarse_sweep).  The coarse chain
 * advances one slice at a time, so its sweeps see only that slice's lines.  STAGED: a CTA copies
 * its lines and their factors into shared memory with asynchronous copies, one thread per line
 * runs the Thomas/LDL^T recurrences there, and the CTA writes back with the correction fused.
 * STREAMED: one thread per line runs them from global memory with its loads issued a chunk
 * ahead.  Both compute the same recurrences with the same roundings (bitwise equal results).
 * On GB300 the streamed form is faster for FP64 (measured): an FP64 FMA's dependent latency is
 * long, and the staged form runs only the lines of its shared-memory tiles per SM, too few
 * independent chains to hide it. */
#define PS_COARSE_SWEEP_AUTO 0
#define PS_COARSE_SWEEP_STAGED 1
#define PS_COARSE_SWEEP_STREAMED 2

typedef struct ps_grid ps_grid;
typedef struct ps_operator ps_operator;
typedef struct ps_splitting ps_splitting;
typedef struct ps_problem ps_problem;

/* Self-test of the device-side wait limit (no counterpart in the paper): launches a kernel
 * that waits, with the bounded wait every tile and DD kernel uses, on a shared-memory
 * barrier that nothing arrives at, for limit_us microseconds (1..1e6).  Returns
 * PS_ERR_DEVICE_TIMEOUT when the wait ran out and the kernel reported it, which is the
 * expected outcome; the CUDA context stays usable.  PS_ERR_INVALID for a bad limit. */
int ps_selftest_wait_timeout(int limit_us, uintptr_t stream);

/* Message of the calling thread's last failed call ("" if none). */
const char* ps_last_error(void);
/* ABI version of this header, major*100 + minor; raised whenever a struct layout or a
 * signature changes.  ps_version() returns the value the library was built with, so a
 * caller can refuse a library built from another header. */
#define PS_VERSION 103
int ps_version(void);

/* ---- grid: unit box, n[d] interior nodes, h_d = 1/(n[d]+1) (Sec. 2.2) ---------------- */
/* dim = 2 or 3; n[0..dim-1] >= 1 (n[2] ignored in 2-D).  PS_ERR_INVALID otherwise. */
int ps_grid_create(int dim, const int n[3], ps_grid** out);
int ps_grid_destroy(ps_grid* g);

/* ---- operator L u = div(a grad u) - c u + f (Sec. 2.1, eq. cont_problem) -------------- */
/* a_nodal_dev: nodal diffusion (boundary included) or NULL for a = 1; must be > 0.
 * c >= 0: reaction.  src_dev: spatial source on interior nodes or NULL (f = 0).
 * src_t_host: time factors f(x,t) = src(x) * src_t[j] at the fine times t_j = j*dt,
 * j = 0..src_t_len-1, or NULL (factor 1).  The arrays are copied; the caller may
 * free them after the call.  The edge coefficient is a_{i+1/2} = (a_i + a_{i+1})/2. */
int ps_operator_create(const ps_grid* g, const double* a_nodal_dev, double c, const double* src_dev,
                       const double* src_t_host, int src_t_len, uintptr_t stream, ps_operator** out);
int ps_operator_destroy(ps_operator* op);
/* Operator with every option (ps_operator_create covers a scalar diffusion and one source):
 *   u_t = div(D grad u) - c u + src(x) src_t(t) + src2(x) src2_t(t),
 * D = a I, or in 2-D the full tensor D = [[a, d12], [d12, a]] of Sec. 5.2 when d12_nodal_dev is
 * given (nodal, boundary included, same layout as a; D must be SPD at every node).  The mixed
 * derivatives make the stencil nine-point: only the DD splitting takes such an operator
 * (ps_splitting_create returns PS_ERR_UNSUPPORTED for PS_SPLIT_DIM, as the paper notes in
 * Sec. 2.1).  The operator is assembled cell by cell: on every grid cell, D is the mean of its
 * four nodal values and the DD weight rho_j is taken at the cell centre; the cell's quadratic
 * form uses the x-differences of its bottom and top edges, the y-differences of its left and
 * right edges and its mean gradient for the d12 term.  With d12 = 0 this is a five-point
 * scheme whose edge coefficient is the mean of the two adjacent cells' a (not the nodal mean of
 * ps_operator_create).  src2 needs src and the DD splitting; src2_t is indexed like src_t.
 * Fields left NULL / 0 are absent (a = 1, d12 = 0, no source). */
typedef struct {
  const double* a_nodal_dev;   /* diagonal diffusion a, nodal, or NULL (a = 1) */
  const double* d12_nodal_dev; /* off-diagonal diffusion, nodal, or NULL (D = a I) */
  double c;                    /* reaction, >= 0 */
  const double* src_dev;       /* first source term, interior nodes, or NULL */
  const double* src_t_host;    /* its time factors at t_j = j dt, or NULL (1) */
  int src_t_len;
  const double* src2_dev;      /* second source term, or NULL */
  const double* src2_t_host;
  int src2_t_len;
} ps_operator_desc;
int ps_operator_create_ex(const ps_grid* g, const ps_operator_desc* desc, uintptr_t stream, ps_operator** out);

/* ---- splitting L = L_1 + ... + L_M (Sec. 2.1) ----------------------------------------- */
typedef struct {
  int boxes[2];   /* boxes per direction (>= 1; a direction with 1 box is not split) */
  double overlap; /* overlap width beta in [0,1] units, centred on every core boundary */
} ps_dd_params;
/* kind = PS_SPLIT_DIM (dd ignored) or PS_SPLIT_DD (2-D only; colours
 * (bx%2, by%2) = (0,0),(1,0),(0,1),(1,1) applied in that order; cos^2 ramps). */
int ps_splitting_create(const ps_operator* op, int kind, const ps_dd_params* dd, ps_splitting** out);
int ps_splitting_destroy(ps_splitting* sp);

/* ---- parareal problem (Sec. 3) ----------------------------------------------------------- */
typedef struct {
  int precision; /* PS_PREC_FP64 or PS_PREC_MIXED */
  int schedule;  /* PS_SCHED_* (other values: PS_ERR_INVALID) */
  int timing;    /* 1: per-phase CUDA events (ps_problem_stats); 2: also per-kernel
                    events (ps_problem_kernel_times) */
  int dd_slices_per_block; /* DD subdomain solves: time slices per CTA (1, 2 or 4); 0 = 2 */
  int tile_positions;      /* fine line solves: line positions per TMA tile (1, 2, 4); 0 = auto
                              (FP32: 1; FP64: as many as fit 96 KB, up to 4) */
  int tile_pipeline;       /* fine line solves: 1 persistent CTAs with a ring of three stages,
                              2 one tile per CTA, 0 = auto (one tile per CTA) */
  int tile_slots;          /* fine line solves: time slices per TMA tile (16, 32, 64); 0 = auto */
  int tol_mode;            /* stopping test: 0 = max_n ||U_n^k - U_n^{k-1}||_inf < tol (absolute);
                              1 = max_n ||U_n^k - U_n^{k-1}||_inf / ||U_n^k||_inf < tol (per slice) */
  int coarse;              /* PS_COARSE_FP64 (0) or PS_COARSE_DELTA32 */
  int tile_lines_per_thread; /* fine line solves (FP32 tiles of 32+ slots): lines a thread solves
                                side by side, 1 or 2; 0 = auto (1) */
  int fine_method;         /* PS_FINE_FIE (0) or PS_FINE_DR */
  int overlap_phases;      /* 1: with the dimensional splitting, the fine phase of an iteration runs on
                              a side stream, slot group by slot group, and the coarse chain follows
                              each group as it finishes (the same values, computed concurrently);
                              0 (default): the fine phase completes before the chain starts.
                              Measured on GB300 at 255^3 x 64 slices, the overlapped order is
                              slower: the half-range tiles fetch whole 256-byte rows and the chain's
                              latency-bound sweeps slow down beside the tiles */
  int coarse_sweep;        /* coarse-propagator line solves on one slice (dimensional splitting):
                              PS_COARSE_SWEEP_STAGED or PS_COARSE_SWEEP_STREAMED; 0 = streamed
                              unless ps_autotune picks staged */
} ps_params;

/* fine, coarse: splittings of the same operator used by F and G (coarse = NULL: use
 * fine).  T > 0; N slices; G = g_steps FIE steps of DeltaT/g_steps; F = f_steps FIE
 * steps of dt = DeltaT/f_steps; f_steps % g_steps == 0.  Builds the substep factors
 * of (I - tau A_j) for both step sizes on the device (FP64) and allocates the slice
 * states: (N+1) U, N F-results, N Gold (PS_COARSE_FP64) or two FP32 single-slice states
 * (PS_COARSE_DELTA32), and the slice-interleaved fine working state (FP32 in
 * PS_PREC_MIXED). */
int ps_problem_create(const ps_splitting* fine, const ps_splitting* coarse, double T, int N, int g_steps,
                      int f_steps, const ps_params* params, uintptr_t stream, ps_problem** out);
int ps_problem_destroy(ps_problem* p);
/* Change the slice count N and the propagators' step counts of an existing problem (Sec. 3:
 * DeltaT = T/N, G = g_steps FIE steps of DeltaT/g_steps, F = f_steps FIE steps of
 * DeltaT/f_steps; same rules as at creation).  Rebuilds the substep factors for the new step
 * sizes and reallocates the slice states; the previous run's states, history and adjoint
 * workspaces are dropped, the tile schedule (ps_autotune) is kept.  PS_ERR_INVALID for bad
 * counts (nothing changed then) or while the problem belongs to a batch; PS_ERR_OOM when the
 * new states do not fit, after which the problem has no slices and refuses every run until a
 * later call succeeds. */
int ps_problem_set_slices(ps_problem* p, int N, int g_steps, int f_steps, uintptr_t stream);

/* Parareal from u0_dev: U_0 = u0, U^0 by a sequential coarse sweep, then
 * U_{n+1}^{k} = F(U_n^{k-1}) + (G(U_n^{k}) - G(U_n^{k-1})) for k = 1, 2, ...
 * Stops at the first k with inc_k = max_{n>=1} ||U_n^k - U_n^{k-1}||_inf < tol, at
 * k = N (then U is the sequential fine solution), or at k = max_iter (<= 0: N).
 * *iters_out = k.  Reaching k = N is not an error.  Slices n < k-1 whose input
 * did not change are not recomputed (their result is bitwise the same). */
int ps_run_parareal(ps_problem* p, const double* u0_dev, double tol, int max_iter, uintptr_t stream,
                    int* iters_out);
/* Same from host memory: copies u0_host in, runs, copies U_N out to uN_host. */
int ps_run_parareal_host(ps_problem* p, const double* u0_host, double* uN_host, double tol, int max_iter,
                         uintptr_t stream, int* iters_out);
/* Copy U_slice (0..N) of the last run to out_dev. */
int ps_get_state(const ps_problem* p, int slice, double* out_dev, uintptr_t stream);
/* inc_k for k = 1..len of the last run; len = min(iterations, cap). */
int ps_get_history(const ps_problem* p, double* inc_host, int cap, int* len);
/* Overwrite U_slice (0..N) with in_dev.  The problem's iterate is then no longer resumable. */
int ps_set_state(ps_problem* p, int slice, const double* in_dev, uintptr_t stream);

/* Checkpoint and resume of a parareal run (no counterpart in the paper).  After
 * ps_run_parareal (or ps_resume_parareal) stopped at iteration k -- at its tolerance or at
 * max_iter -- ps_checkpoint_save writes k, the history inc_1..inc_k, the slice states U^k and,
 * with the FP64 coarse propagator, the coarse values G(U_n^k) that the next correction
 * subtracts, into host memory (ps_checkpoint_bytes gives the size).  ps_checkpoint_load puts
 * them into a problem of the same grid, slice count and coarse form (PS_ERR_INVALID
 * otherwise), and ps_resume_parareal continues with iteration k+1 to the given tolerance or
 * max_iter (counted from the start of the run; <= 0: N).  The continued run computes exactly
 * the values the uninterrupted run computes.  A run that had already met `tol` does not
 * iterate further.  ps_resume_parareal also continues the problem's own stopped run.  The
 * adjoint, ps_set_state, ps_problem_set_slices and ps_problem_update_coefficients end the
 * resumability of the current iterate. */
int ps_checkpoint_bytes(const ps_problem* p, size_t* bytes);
int ps_checkpoint_save(const ps_problem* p, void* host_buf, size_t bytes, uintptr_t stream);
int ps_checkpoint_load(ps_problem* p, const void* host_buf, size_t bytes, uintptr_t stream);
int ps_resume_parareal(ps_problem* p, double tol, int max_iter, uintptr_t stream, int* iters_out);

/* Sequential fine solution (the plain comparator): U_out_dev gets (N+1) states at T_n. */
int ps_run_fine_sequential(ps_problem* p, const double* u0_dev, double* U_out_dev, uintptr_t stream);
/* Sequential coarse solution U_n = G^n(u0), (N+1) states. */
int ps_run_coarse_sequential(ps_problem* p, const double* u0_dev, double* U_out_dev, uintptr_t stream);

/* Replace the nodal diffusion coefficient (same layout as at ps_operator_create, which must
 * have been given one) and rebuild the problem's substep factors for both step sizes.  The
 * operator is shared: other problems built on it see the new coefficient after their own
 * update call. */
int ps_problem_update_coefficients(ps_problem* p, const double* a_nodal_dev, uintptr_t stream);

/* Vector-Jacobian product of the last parareal run (no counterpart in the paper; the
 * transpose of the FIE steps).  With U_N the sequential fine solution from u0 and the
 * coefficient a, and g = gN_dev an upstream gradient dL/dU_N, returns dL/du0 = J_u0^T g and
 * dL/da = J_a^T g (nodal, boundary included; NULL to skip).  The slice-boundary adjoints
 * lambda_n = F^T lambda_{n+1}, lambda_N = g, come from a parareal iteration with the
 * transposed propagators (substeps in reverse order, no source) run backwards in time to
 * the per-slice relative tolerance `tol` (max_iter <= 0: N); the coefficient gradient then
 * recomputes the fine steps inside every slice from the forward checkpoints U_n (all slices
 * at once, FP64) and accumulates -tau (nu_Q - nu_P)(w_Q - w_P)/h^2 over every edge of every
 * substep, half to each end node.  Needs a preceding ps_run_parareal on this problem (its
 * states are the checkpoints, so run it to a tight tolerance, e.g. tol_mode = 1).  dL/du0
 * is available in every FIE form (FP64 or FP32 fine line solves, dimensional or DD
 * splitting, FP64 coarse propagator); the coefficient gradient needs FP64 precision and the
 * dimensional splitting, the increment-form coarse propagator and DR fine steps are refused
 * (PS_ERR_UNSUPPORTED).  The problem's states are the forward ones again on return;
 * *iters_out = adjoint parareal iterations. */
int ps_adjoint_vjp(ps_problem* p, const double* gN_dev, double tol, int max_iter, double* grad_u0_dev,
                   double* grad_a_dev, uintptr_t stream, int* iters_out);
/* Gradient of the loss J = 1/2 ||U_N - u_target||^2 (sum over interior nodes) of the last
 * parareal run: ps_adjoint_vjp with the upstream gradient g = U_N - u_target, formed on the
 * device.  *J_out (host, may be NULL) receives J, summed in a fixed order (the same value on
 * every call with the same data).  Same requirements and errors as ps_adjoint_vjp. */
int ps_adjoint(ps_problem* p, const double* u_target_dev, double tol, int max_iter, double* grad_u0_dev,
               double* grad_a_dev, uintptr_t stream, double* J_out, int* iters_out);

/* Sequential coarse solution U_n = G^n(u0) without allocating any device memory.
 *
 * No counterpart in the paper: this is a service for callers that cannot allocate, such as
 * code running where cudaMalloc is forbidden or unsafe (inside a host callback or a memory
 * pool's own allocation hook, or under a budget that leaves no device memory to spare).
 * It computes exactly what ps_run_coarse_sequential computes (same kernels, same order),
 * but keeps the coarse working state in a fixed array of PS_NOALLOC_MAX_UNKNOWNS doubles
 * (8 MiB) that every GPU loading this library reserves until the process exits, instead of
 * in the problem's own workspace.  The caller passes the input u0_dev and the output
 * U_out_dev ((N+1) states), as for the allocating version.
 *  - Grids with more than PS_NOALLOC_MAX_UNKNOWNS interior unknowns are rejected with
 *    PS_ERR_INVALID before any GPU work.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 *    with that device current.
 *  - Like the allocating version, the call waits for `stream` before it returns: it reads the
 *    device-side error flag of its kernels back to the host.
 *  - All calls share the one array: calls that overlap on the GPU (other streams, other
 *    threads) race and produce wrong results.  Serialise them.
 *  - Nothing in the array needs to start at zero: each coarse step overwrites it fully. */
#define PS_NOALLOC_MAX_UNKNOWNS (1 << 20)
int ps_run_coarse_sequential_noalloc(ps_problem* p, const double* u0_dev, double* U_out_dev, uintptr_t stream);

/* Building blocks on one state x_dev (in place), for testing the kernels.
 * which = 0: fine propagator's step size and splitting, 1: coarse.
 * ps_substep_solve: x <- (I - tau A_m)^{-1} x (one internal stage of eq. FIE_method).
 * ps_propagate: nsteps FIE steps (also when params.fine_method is PS_FINE_DR); step q ends at
 * fine time index t0 + (q+1)*tstride. */
int ps_substep_solve(ps_problem* p, int which, int m, double* x_dev, uintptr_t stream);
int ps_propagate(ps_problem* p, int which, int nsteps, int t0, int tstride, double* x_dev, uintptr_t stream);

typedef struct {
  int iterations;          /* k of the last run */
  double unknown_updates;  /* interior unknowns advanced by one FIE step, summed over the run */
  double ms_total;         /* device time of the last run (events; timing != 0) */
  double ms_fine;          /* of which F phases */
  double ms_coarse;        /* of which the initial sweep, G phases and corrections */
  int kernel_launches;     /* kernels this library launched in the last run */
} ps_stats;
int ps_problem_stats(const ps_problem* p, ps_stats* out);

/* Per-kernel-kind device times of the last run, recorded when params.timing >= 2 with a
 * CUDA event pair around every launch on the run's stream.  name: "<phase>.<axis>.<type>"
 * (phase F = fine, G = coarse; +corr / +init when the parareal correction / initial sweep
 * is fused in, +dcorr for the correction of the FP32 coarse increment form).  bytes / flops: algorithmic traffic and FP work summed over the launches
 * (each sweep reads its right-hand side and writes its result once, reads the factors once
 * per launch; 5 flops per unknown per sweep, FMA = 2).  len = number of kinds (<= cap). */
typedef struct {
  char name[32];
  int launches;
  double ms;
  double bytes;
  double flops;
} ps_kernel_time;
int ps_problem_kernel_times(const ps_problem* p, ps_kernel_time* out, int cap, int* len);

/* ---- batches of independent problems (uneven grids, slice and step counts) ------------- */
/* A batch advances its problems' parareal iterations together: every phase-step of an
 * iteration is one grouped persistent launch over all problems that still iterate (the fine
 * line solves of every slice of every problem, then each coarse step with its correction),
 * the whole iteration is one CUDA graph replayed until every problem has converged, and only
 * small work tables change between replays.  Results equal each problem's own
 * ps_run_parareal bitwise.  Problems: all 2-D or all 3-D, dimensional splitting, PS_PREC_MIXED, one coarse
 * step per slice, with or without a source term, all with the same coarse form (PS_COARSE_FP64,
 * or PS_COARSE_DELTA32 with rows of at most 1024 nodes) and the default coarse x-sweep
 * schedule of that form, all with a nodal coefficient or all without (PS_ERR_UNSUPPORTED
 * otherwise).  The batch keeps pointers to the problems
 * (destroy it first); states and histories are read per problem afterwards (ps_get_state,
 * ...).  While a problem belongs to a batch, ps_autotune only considers the tile shapes
 * the batch's grouped kernels run (one tile per work item, one line per thread, one line
 * position per tile).  From those, each ps_batch_run derives the batch's own tile shapes:
 * every tile of a launch reserves as much shared memory as the batch's largest, and
 * problems with shorter lines take up to four line positions per tile to fill it (the
 * problems' own plans, and every result, stay as they are). */
typedef struct ps_batch ps_batch;
/* count >= 0 problems (problems may be NULL when count = 0); more join with ps_batch_add. */
int ps_batch_create(ps_problem* const* problems, int count, uintptr_t stream, ps_batch** out);
/* Append problem p (same requirements as at creation; PS_ERR_UNSUPPORTED otherwise, the batch
 * unchanged).  Its index is the number of problems the batch held before the call. */
int ps_batch_add(ps_batch* b, ps_problem* p, uintptr_t stream);
/* Copy state U_slice (0..N_p) of problem `index` of the last ps_batch_run to out_dev. */
int ps_batch_get_state(const ps_batch* b, int index, int slice, double* out_dev, uintptr_t stream);
/* u0_devs: host array of `count` device pointers.  Each problem stops at the first k with
 * max_n ||U_n^k - U_n^{k-1}||_inf < tol, at k = N_p, or at max_iter (<= 0: no cap).
 * iters_out (host, `count` ints, may be NULL) receives each problem's k. */
int ps_batch_run(ps_batch* b, const double* const* u0_devs, double tol, int max_iter, uintptr_t stream,
                 int* iters_out);  /* PS_ERR_INVALID for an empty batch */
/* iterations = the largest k, unknown_updates over all problems, kernel_launches (graph nodes
 * executed).  ms fields are 0. */
int ps_batch_stats(const ps_batch* b, ps_stats* out);
const char* ps_batch_last_error(void);
int ps_batch_destroy(ps_batch* b);

/* Autotuner of the line-solve schedules: times the fine sweeps of this problem with each
 * candidate tile shape (time slices per tile 16/32/64, line positions 1/2, lines per thread
 * 1/2, one tile per CTA or a persistent ring of three shared-memory stages) for about
 * budget_ms and installs the fastest; with the dimensional splitting it also times the coarse
 * x-sweep's schedules (PS_SCHED_*) and one coarse step's sweeps staged and streamed
 * (PS_COARSE_SWEEP_*) and installs the fastest of each.  The tile shapes and the staged/
 * streamed choice change no result (the same arithmetic per line); the x-sweep schedule
 * changes the coarse values at rounding level (see PS_SCHED_*), so for a problem that belongs
 * to a batch with the FP64 coarse propagator only Thomas is considered.  *choice_out (may be
 * NULL) receives coarse_sweep*100000 + lines_per_thread*10000 + slots*100 + positions*10 +
 * pipelined; ps_params.schedule of the problem holds the x-sweep's choice.  With the DD
 * splitting (FIE fine steps) it times the fine colour solves with 1, 2 and 4 time slices per
 * CTA instead and installs the fastest as dd_slices_per_block (*choice_out = that count; the
 * same arithmetic per slice in every case). */
int ps_autotune(ps_problem* p, int budget_ms, uintptr_t stream, int* choice_out);
/* The timing record of the last ps_autotune on this problem: one entry per candidate timed,
 * name "fine:<slots>x<positions>/v<lines per thread>/<tile|ring>", "coarse:<staged|streamed>",
 * "coarse-x32:<thomas|pcr|hybrid>" (increment form) or "coarse-x64:<thomas|hybrid>",
 * "coarse-corr:<fused|split>" (FP64 coarse form: the correction in the last sweep's epilogue or
 * as its own pass; the same values either way), "dd:<S>-slices-per-cta" (DD), and its
 * time per candidate run (ms; fine: the sweeps of all directions over all slices; coarse: one
 * coarse step's sweeps; coarse-x*: one x-sweep).
 * chosen = 1 for the installed candidate of each group.  len = number of entries (<= cap). */
typedef struct {
  char name[48];
  double ms;
  int chosen;
} ps_tune_entry;
int ps_autotune_record(const ps_problem* p, ps_tune_entry* out, int cap, int* len);
/* Same schedule on `dst` as on `src` (same grid and slice count). */
int ps_copy_schedule(const ps_problem* src, ps_problem* dst);

#ifdef __cplusplus
}
#endif
#endif /* PS_H */
