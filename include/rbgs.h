/*
 * rbgs.h -- C ABI of librbgs.so: red-black Gauss-Seidel (RBGS) for the 2D Poisson
 * equation on GB300 (sm_103a).
 *
 * The method (Section 2 of "Exploiting Task-Based Parallelism for the Red-Black
 * Gauss-Seidel Method on 2D Grids", Long, Ramirez-Hidalgo, Frommer, Pleiter):
 *   -Lap u = f on the unit square, u = g on the boundary (the paper writes Lap u = f;
 *   this is the same problem with f -> -f), uniform grid h = 1/(N+1), and the 5-point
 *   update of Eq. (1),
 *       u_ij <- (h^2 f_ij + u_{i-1,j} + u_{i+1,j} + u_{i,j-1} + u_{i,j+1}) / 4,
 *   applied first to every red point (i + j even) and then to every black point
 *   (i + j odd); one red+black pair is one sweep (Algorithms 1 and 2).
 *
 * Arithmetic: every update is evaluated as (((h2*f + N) + S) + W) + E, times 0.25, with
 * each operation correctly rounded and h2*f never contracted into an add (h2*f is formed
 * once, when a problem is loaded).  The FP64 adds run as fused multiply-adds by 1.0, which
 * round the exact sum once, the same value as the add; x0.25 is an exact exponent step.
 * So the FP64 path gives the same bits as a plain sequential C loop in that order.
 *
 * Grids, all row-major, i = row (x, slow), j = column (y, fast):
 *   f      N x N interior values (f_ij at index (i-1)*N + (j-1)), float64
 *   u      (N+2) x (N+2) including the Dirichlet ring (u_ij at index i*(N+2) + j);
 *          the ring holds g and stays fixed, the interior is the iterate
 * Pointers may address device memory or host memory (pageable or pinned); the library
 * copies through the CUDA runtime with unified addressing.  The caller keeps ownership
 * of everything it passes; the library owns the buffers inside a context.
 *
 * Errors: every call returns an rbgs_status; nothing is thrown across the ABI.  On a
 * non-OK status rbgs_last_error() returns a message for the calling thread.  CUDA
 * errors from a failed launch leave the context usable only for rbgs_destroy.
 * Work is ordered on the stream given at creation (NULL = the legacy default stream);
 * calls that return a host scalar synchronise that stream.
 *
 * Devices and threads: a context lives on the device that is current when rbgs_create
 * runs; call it with that device current (the library does not switch devices).  Calls
 * on one context must not overlap in time; separate contexts may be used from separate
 * threads at once.
 */
#ifndef RBGS_H
#define RBGS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rbgs_ctx *rbgs_t;

typedef enum {
    RBGS_OK = 0,
    RBGS_EINVAL = 1,      /* bad argument: null pointer, n < 1, h2 <= 0, bad option     */
    RBGS_ENOMEM = 2,      /* device or pinned host allocation failed                     */
    RBGS_ECUDA = 3,       /* a CUDA runtime/driver call failed                           */
    RBGS_ENOTCONV = 4,    /* max_sweeps reached, or the residual stalled (stall_checks);
                             the iterate is kept                                          */
    RBGS_ENONFINITE = 5,  /* the residual became NaN or Inf                              */
    RBGS_ETIMEOUT = 6     /* a bounded device-side wait gave up: the grid barrier of the
                             cooperative FP64 launch or the TMA wait of the temporal
                             kernel (reported by the next rbgs_residual or rbgs_solve).
                             Sticky: the iterate is left part-updated and every later
                             rbgs_residual / rbgs_solve on the context returns it again;
                             destroy the context.  In rbgs_solve_batched: the batch's
                             device-time budget (max_seconds) ran out for that problem    */
} rbgs_status;

typedef enum {
    RBGS_FP64 = 0,        /* plain FP64 sweeps                                            */
    RBGS_FP32_REFINE = 1  /* FP32 sweeps on the defect equation + FP64 residual/correction */
} rbgs_precision;

typedef enum {
    RBGS_KERNEL_AUTO = 0,     /* FP64 sweeps: PERSISTENT for 416 <= n <= 32768 with the default
                                 launch-shape options, else COLOUR.  FP32 inner sweeps of
                                 RBGS_FP32_REFINE: WAVEFRONT (depth 4) when n > 2048 and
                                 tblock_k = 0, else COLOUR                                   */
    RBGS_KERNEL_COLOUR = 1,   /* one launch per colour (half-sweep kernels)               */
    RBGS_KERNEL_TEMPORAL = 2, /* several sweeps per shared-memory tile, halo recompute      */
    RBGS_KERNEL_WAVEFRONT = 3,/* several sweeps per pass, a register wavefront per strip   */
    RBGS_KERNEL_PERSISTENT = 4/* FP64 sweeps: all of an rbgs_sweep call in one cooperative
                                 launch, a bounded grid barrier between the colours
                                 (n <= 32768; the launch-shape options do not apply).  FP32
                                 inner sweeps: as COLOUR                                     */
} rbgs_kernel;

typedef struct {
    int precision;     /* rbgs_precision                                                  */
    int kernel;        /* rbgs_kernel                                                     */
    int check_every;   /* sweeps between residual checks in rbgs_solve (0: 100)            */
    long max_sweeps;   /* rbgs_solve gives up after this many sweeps (0: 1e9)              */
    int tblock_k;      /* sweeps per pass: RBGS_KERNEL_TEMPORAL 1, 2, 4 (FP64) or 2, 4, 8
                          (FP32 inner sweeps); RBGS_KERNEL_WAVEFRONT 2, 4 (FP64) or 2, 4, 6
                          (FP32 inner sweeps); 0: automatic                                */
    int tile_rows;     /* rows per thread block (0: automatic)                             */
    int fp64_emulate;  /* FP64 adds issued on the integer pipe per 8 (-1: automatic)       */
    int inner_sweeps;  /* FP32 sweeps per defect correction for RBGS_FP32_REFINE (0: auto) */
    int sweep_values;  /* values each thread updates per row in a half-sweep: 2 or 4 (0: auto) */
    int sweep_rows;    /* rows each thread updates per loop step in a half-sweep: 1 or 2 (0: auto) */
    int int_rows;      /* FP64 hybrid half-sweep: between strips of tile_rows rows whose adds run on
                          the FP64 pipe, strips of int_rows rows whose adds run as exact integer
                          IEEE additions (same results; 0: off, -1: automatic)                  */
    int team_size;     /* rbgs_solve_batched: 2 or 4 forces the phased plan, in which the largest
                          problems left over after full waves of one block per problem are each
                          solved by a thread-block cluster of team_size blocks; 1: one block per
                          problem always; 0: the autotuner decides                              */
    int fma;           /* FP64 update of rbgs_sweep / rbgs_solve (RBGS_FP64 only):
                          0 (default): bit-exact, (((h2f + N) + S) + W) + E times 0.25 with every
                            step correctly rounded, the same bits as the plain sequential loop;
                          1: fused, one rounding per update instead of four: the five terms are
                            summed exactly in 64-bit fixed point (scale 2^e, chosen before each
                            block of at most 1024 sweeps from max|u| and max|h2 f| so that no sum
                            can overflow; terms are truncated to multiples of 2^-e) and the sum
                            divided by 4 is rounded once to binary64 (nearest, ties to even).
                            Integer arithmetic only, so the update leaves the FP64 pipe.  Agrees
                            with the bit-exact iterate to <= 1e-13 relative max-norm after the same
                            sweeps (the tolerance set for this mode); a non-finite value in u or h2 f makes
                            that block of sweeps run the bit-exact update.  One launch per colour
                            (the kernel option does not apply)                                   */
    int stall_checks;  /* rbgs_solve and rbgs_solve_batched stop a problem with RBGS_ENOTCONV when
                          its residual has not reached a new minimum for this many consecutive
                          checks (0: 64; -1: never), so a tolerance below the rounding floor
                          does not sweep until max_sweeps                                        */
    double max_seconds;/* rbgs_solve_batched: device-time budget of the whole batch in seconds,
                          measured from the first problem's start (%globaltimer); a problem still
                          running, or not yet started, when it is spent ends with RBGS_ETIMEOUT
                          and keeps its iterate (0: no budget)                                   */
} rbgs_opts;

/* Fills *opts with the defaults (all automatic).  Not in the paper: library mechanics. */
void rbgs_default_opts(rbgs_opts *opts);

/*
 * Creates a solver for one N x N problem (Section 2 and Eq. (1): h = 1/(N+1); the inputs
 * of Algorithm 1, grid, f and h, with the ring of the Dirichlet problem; the caller passes
 * h2 = h*h as it wants it rounded).  f: N*N values; u_init: (N+2)^2 values with the
 * Dirichlet ring and the initial guess.  opts may be NULL (defaults).  The stream is a
 * cudaStream_t (NULL: legacy default stream).  On success *out owns device buffers of
 * about 4 (N+2)^2 doubles (plus FP32 copies for RBGS_FP32_REFINE).
 */
rbgs_status rbgs_create(int n, double h2, const double *f, const double *u_init,
                        const rbgs_opts *opts, void *cuda_stream, rbgs_t *out);

/* nsweeps red+black sweeps of Eq. (1) (Algorithm 1's iteration; nsweeps >= 0). Async. */
rbgs_status rbgs_sweep(rbgs_t ctx, long nsweeps);

/*
 * Not in the paper, which fixes the iteration count (Section 4): the convergence measure
 * the library adds.  Relative residual rho = ||b - A u||_2 / ||b||_2 of the current iterate, with
 * A = (4 I - neighbours)/h^2 and b = f plus the ring terms / h^2 (the linear system of
 * Eq. (1)); rho = ||b - A u||_2 * h^2 when b = 0.  Synchronises the stream.
 * Right after rbgs_sweep (nsweeps > 0) only the red points are summed: the black points'
 * residual is exactly zero then, so rho is the same, bit for bit, at half the cost.
 * Returns RBGS_ENONFINITE (and writes rho) when rho is NaN or Inf.
 */
rbgs_status rbgs_residual(rbgs_t ctx, double *rel);

/*
 * Sweeps of Eq. (1) until rho <= tol.  The paper runs a fixed number of iterations
 * (Section 4); this stopping rule is the library's.  Evaluates rho before the first sweep
 * and then every check_every sweeps.  *sweeps_done gets the sweeps performed, *rel the last rho
 * (either may be NULL).  RBGS_ENOTCONV after max_sweeps or when rho has stalled
 * (opts.stall_checks), RBGS_ENONFINITE on NaN/Inf.
 */
rbgs_status rbgs_solve(rbgs_t ctx, double tol, long *sweeps_done, double *rel);

/* Copies the current iterate, ring included, into u_out ((N+2)^2 values: the grid of
 * Section 2).  Not in the paper: library mechanics. */
rbgs_status rbgs_get_solution(rbgs_t ctx, double *u_out);

/* Replaces the iterate and the ring by u_in ((N+2)^2 values), e.g. to resume a run.  Not
 * in the paper: library mechanics. */
rbgs_status rbgs_set_solution(rbgs_t ctx, const double *u_in);

/*
 * Not in the paper: library mechanics.  Loads a new problem of the same N and h2 into ctx: f (N*N values) and u_init ((N+2)^2
 * values, ring and initial guess), host or device memory, as rbgs_create reads them.  The
 * context's device buffers, options and cached launch graphs are kept, so a stream of
 * problems of one size needs no allocation after the first.  The result is the same as
 * rbgs_destroy followed by rbgs_create with these inputs.  Synchronises the stream (the
 * right-hand side norm is read back).
 */
rbgs_status rbgs_set_problem(rbgs_t ctx, const double *f, const double *u_init);

/*
 * Not in the paper: library mechanics for serving a stream of problems of the context's
 * size (same N and h2; each is Section 2's problem, swept by Eq. (1)).  For problem
 * q = 0 .. count-1, in order: load f[q] and u_init[q] (as rbgs_set_problem), nsweeps
 * sweeps (as rbgs_sweep, with the context's options), the residual rho[q] (as
 * rbgs_residual; rho may be NULL) and the solution into u_out[q] (as rbgs_get_solution).
 * Host buffers move on the library's own copy streams, one per direction, through
 * double-buffered device staging: problem q+1's inputs and problem q-1's solution travel
 * while problem q sweeps.  With page-locked host memory (cudaHostAlloc or registered) the
 * copies run asynchronously; pageable memory works, but its copies hold the calling thread.
 * Device buffers are used in place.  The staging (two natural-layout copies of f and u_init
 * and two of u_out, for the directions that see host memory) is allocated on first use and
 * kept with the context.  Returns once every solution is in place; work the caller queues
 * on the context's stream afterwards follows all of it.  RBGS_ENONFINITE when some rho is
 * not finite (every output is still written); the context then holds the last problem.
 * RBGS_FP64 contexts only (fma 0 or 1).
 */
rbgs_status rbgs_run_stream(rbgs_t ctx, int count, const double *const *f, const double *const *u_init,
                            long nsweeps, double *const *u_out, double *rho);

/* Problem n of a batch: interior size, h^2, f (N*N) and u_init ((N+2)^2). */
typedef struct {
    int n;
    double h2;
    const double *f;
    const double *u_init;
} rbgs_problem;

/* Per-problem outcome of rbgs_solve_batched. */
typedef struct {
    int status;          /* rbgs_status of this problem                                   */
    long sweeps;         /* sweeps performed                                              */
    double rel;          /* final relative residual                                       */
    double latency_ms;   /* device time from the batch start to this problem's completion  */
} rbgs_result;

/*
 * Not in the paper: the batched growth direction, many independent problems of Section 2
 * (each swept by Eq. (1), red then black) in persistent launches.
 * Solves nprob independent problems of uneven sizes (1 <= N_p <= 32768) to rho <= tol each,
 * in persistent launches captured with the packing and unpacking in a CUDA graph.  A
 * thread block claims one problem at a time, largest first, and solves it on its own
 * (FP64 sweeps with a residual check every opts->check_every sweeps, or, with
 * RBGS_FP32_REFINE, the mixed-precision refinement with opts->inner_sweeps FP32 sweeps per
 * correction), so each problem's iterate equals a single-problem solve with the same
 * options.  In the phased plan (opts->team_size) the largest problems that would otherwise
 * run in a last, partly filled wave are each solved by a cluster of 2 or 4 blocks on as many
 * SMs, with the same iterate.  The launch shape (threads per block, blocks per SM, team
 * size) is picked by a built-in autotuner on first use for a given size mix, unless
 * opts->team_size (> 1), or opts->tile_rows (> 0: 256, 512 or 1024 threads) and
 * opts->tblock_k (blocks per SM), fix it.  u_out[p] receives problem p's
 * solution ((N_p+2)^2 values, device or host memory); res[p] its outcome, latency_ms
 * measured on the device from the batch's first problem start to this problem's end.
 * A problem whose rho stops reaching new minima for opts->stall_checks checks ends with
 * RBGS_ENOTCONV; once opts->max_seconds of device time have passed since the batch's
 * first problem started, every problem still running or not yet started ends with
 * RBGS_ETIMEOUT (both keep the iterate reached).
 * Returns RBGS_OK when every problem converged, else the first failing status.
 * Synchronises the stream.
 */
rbgs_status rbgs_solve_batched(int nprob, const rbgs_problem *probs, double tol,
                               const rbgs_opts *opts, void *cuda_stream, double **u_out,
                               rbgs_result *res);

/*
 * Not in the paper: library mechanics.
 * Launch shape of the last rbgs_solve_batched call on this thread (zeros before the first):
 * threads per block, blocks per SM, team size (1: one block per problem; 2 or 4: the phased
 * plan), and for the phased plan the number of largest problems solved one per block in its
 * first phase and the number solved by clusters in its second.  Any pointer may be NULL.
 */
void rbgs_batched_last_shape(int *threads, int *blocks_per_sm, int *team, int *first, int *nteam);

/*
 * Relative residual of a natural-layout iterate without allocating memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate device memory
 * (a fixed memory budget set at start-up, code running inside an allocator callback, or
 * code that must avoid the device synchronisation cudaMalloc/cudaFree may imply).
 * f (N*N), u ((N+2)^2, ring included) and rel_out (one double) must be device memory of
 * the current device; rho is written to *rel_out asynchronously on the stream, with the
 * same definition as rbgs_residual.  Its scratch is a fixed array inside the library's
 * device image (128 KiB, held on every GPU that loads the library until the process
 * exits), so N <= 32768; larger N returns RBGS_EINVAL.  The first call on each device looks
 * up that array's device address (and the first call after a cudaDeviceReset of that
 * device looks it up again); make that first call before any stream capture.  Calls share
 * the array: calls that overlap on the GPU race.  No cudaMalloc/cudaFree is made.
 * Nothing is read back, so there is no RBGS_ENONFINITE here: a NaN or Inf in u or f gives
 * a NaN or Inf in *rel_out, which the caller must test (rbgs_residual, by contrast, returns
 * RBGS_ENONFINITE).  The library cannot see the buffers' sizes: f must hold N*N and u
 * (N+2)^2 values (the Python binding checks this before the call).
 */
rbgs_status rbgs_residual_static(int n, double h2, const double *f, const double *u,
                                 double *rel_out, void *cuda_stream);

/* Frees the context (NULL is ignored). Synchronises its stream first.  Not in the paper:
 * library mechanics. */
void rbgs_destroy(rbgs_t ctx);

/* Message for the last non-OK status returned on this thread ("" if none).  Not in the
 * paper: library mechanics. */
const char *rbgs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RBGS_H */
