/*
 * ftgcr.h - C ABI of the GB300-native FT-GCR(k) solver library (libftgcr.so).
 *
 * FT-GCR(k) is the preconditioned generalised conjugate residual method with
 * soft-fault detection and recovery of Gillard & Benacchio, "FT-GCR: a
 * fault-tolerant generalized conjugate residual elliptic solver"
 * (arXiv 2103.07210): Algorithm 1, Section 2.  The library solves the
 * elliptic problem L(phi) = R of Eq. (1) on a regular latitude-longitude grid:
 *
 *   (L phi)_{j,i} = Tx_{j,i}(phi_{j,i+1}-phi_{j,i}) + Tx_{j,i-1}(phi_{j,i-1}-phi_{j,i})
 *                 + Ty_{j,i}(phi_{j+1,i}-phi_{j,i}) + Ty_{j-1,i}(phi_{j-1,i}-phi_{j,i})
 *                 - mu A_j phi_{j,i}
 *
 * the area-integrated finite-volume form of div(D grad phi) - mu phi on the
 * unit sphere (2-D stand-in for the 3-D potential-flow problem of Section 3,
 * Eq. (3)): cell centres theta_j = -pi/2 + (j+1/2) pi/nlat, lambda_i =
 * (i+1/2) 2pi/nlon; Tx_{j,i} = (D_{j,i}+D_{j,i+1})/2 * dth/(cos theta_j dlam),
 * Ty_{j,i} = (D_{j,i}+D_{j+1,i})/2 * cos theta_{j+1/2} dlam/dth, zero flux
 * through the pole faces, A_j the exact cell area.  The left preconditioner
 * ("bespoke", Section 2) is the zonal line operator: the longitude couplings
 * of L plus the diagonal of the rest, one periodic tridiagonal solve per row.
 *
 * Conventions for every entry point:
 *  - Arrays are row-major [nlat][nlon] (longitude fastest), FP64, N = nlat*nlon.
 *  - Unless stated otherwise a pointer may be host or device memory; the
 *    library detects which (cudaPointerGetAttributes).  Host arrays are staged
 *    through buffers owned by the handle.
 *  - The caller owns every array it passes; the handle owns all solver state,
 *    which stays resident on the device between solves.
 *  - Every function returns an int status: 0 (FTGCR_OK), a positive warning,
 *    or a negative error; ftgcr_error_string() names it.  A handle is not
 *    thread-safe: one solve at a time per handle.
 */
#ifndef FTGCR_H
#define FTGCR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FTGCR_OK 0
#define FTGCR_NOT_CONVERGED 1   /* step limit reached; x holds the last iterate */
#define FTGCR_ERR_ARG (-1)      /* bad size, k, tol, pointer, fault or non-finite input */
#define FTGCR_ERR_OOM (-2)      /* device allocation failed */
#define FTGCR_ERR_CUDA (-3)     /* a CUDA call failed (launch, copy, ...) */
#define FTGCR_ERR_TIMEOUT (-4)  /* an in-kernel grid barrier gave up waiting */
#define FTGCR_ERR_BUDGET (-5)   /* serving: request larger than the memory budget */
#define FTGCR_ERR_STATE (-6)    /* call out of order (e.g. stats before any solve) */
#define FTGCR_PENDING 2         /* serving: the request has not finished yet */

/* ---- precision of the iteration ---- */
#define FTGCR_FP64 0  /* every vector, stencil, preconditioner and reduction in FP64 */
#define FTGCR_MIXED 1 /* FP32 inner FT-GCR vectors, stencil, preconditioner and axpys;
                         FP64 inner products (exact FP32 products, float-float per
                         thread, FP64 across threads), FP64 norm test and FP64
                         outer iterative-refinement residual R - L(x) */

/* ---- preconditioner ---- */
#define FTGCR_PRECOND_LINE 0     /* zonal periodic line solve (default) */
#define FTGCR_PRECOND_JACOBI 1   /* diagonal of L */
#define FTGCR_PRECOND_IDENTITY 2 /* no preconditioning */

/* ---- vectors a fault may hit (Algorithm 1 names) ---- */
#define FTGCR_VEC_X 0  /* phi^nu   */
#define FTGCR_VEC_R 1  /* r^nu     */
#define FTGCR_VEC_P 2  /* p^nu     */
#define FTGCR_VEC_AP 3 /* L(p^nu)  */
#define FTGCR_VEC_E 4  /* e = P^-1(r^{nu+1}), the paper's injection site (Section 3) */

typedef struct ftgcr_handle ftgcr_handle;

typedef struct {
  int32_t nlon;      /* >= 3; one latitude row with its two halo rows (and, for the
                        mixed path's line preconditioner, their factors) must fit in
                        one SM's shared memory: nlon <= about 8190 (FTGCR_FP64; beyond
                        about 2150 its line solve reads the factors from global
                        memory) or 8500 (FTGCR_MIXED; beyond about 4350 only with
                        split rounds, see FTGCR_FLAG_SPLIT_ROUNDS), else FTGCR_ERR_ARG */
  int32_t nlat;      /* >= 1 */
  double mu;         /* Helmholtz coefficient per unit area, >= 0 (mu > 0 makes -L definite) */
  int32_t precision; /* FTGCR_FP64 | FTGCR_MIXED */
  int32_t precond;   /* FTGCR_PRECOND_* */
  int64_t max_steps; /* executed-step limit; 0 = 100*ceil(sqrt(N)) + 100 */
  int32_t tiles;     /* row bands per solve (work items per phase); 0 = automatic */
  double inner_tol;  /* FTGCR_MIXED only: relative tolerance of each inner FP32 solve;
                        0 = 1e-5 */
  int32_t max_outer; /* FTGCR_MIXED only: refinement sweeps limit; 0 = 40 */
  int32_t flags;     /* FTGCR_FLAG_* */
} ftgcr_grid;

/* Run plain GCR(k), the paper's unprotected baseline (Section 3): no fault
 * test, so no backup restore (and, in the mixed path, no rejection of
 * refinement updates).  Faults still fire. */
#define FTGCR_FLAG_UNPROTECTED 1
/* FTGCR_MIXED with the line preconditioner: how a step's rounds are laid out.
 * By default a solve whose row bands shared memory cuts below three rows
 * (wide rows: the line-solve constants fill it) runs split rounds: its
 * tiles first form e on their own rows only, and after a grid barrier form
 * L(e) and the dots from e with its halo rows, instead of recomputing two
 * halo rows of e per tile.  These flags force one layout or the other
 * (results differ only by rounding; both are deterministic); both together,
 * or FTGCR_FLAG_SPLIT_ROUNDS on another precision or preconditioner, are
 * FTGCR_ERR_ARG. */
#define FTGCR_FLAG_SPLIT_ROUNDS 2
#define FTGCR_FLAG_FUSED_ROUNDS 4
/* FTGCR_MIXED with the line preconditioner: streamed step rounds, the
 * default for solves of at least 4 Mi points (their Krylov vectors far
 * outgrow the L2 cache).  Each CTA takes one tall band of rows (one band per
 * SM) and walks it row by row: the step's axpy, the row's line solve and the
 * stencil of the row below it, with every operand row staged into shared
 * memory by asynchronous copies issued ahead of the arithmetic.  Only a
 * band's first and last rows wait for a neighbouring band's e, in a second
 * pass.  Needs nlon a multiple of 4; with FTGCR_FLAG_SPLIT_ROUNDS or
 * FTGCR_FLAG_FUSED_ROUNDS, another precision or preconditioner, or rows too
 * wide for the ring of shared-memory slots a step needs: FTGCR_ERR_ARG. */
#define FTGCR_FLAG_STREAMED_ROUNDS 8
/* FTGCR_FP64: take the oracle's operation order where the default takes a
 * faster one that rounds differently.  (1) Inner products: by default each
 * thread sums its products with one fma per element (double-double from the
 * warp up); with this flag every product and partial sum is compensated
 * (Dot2, Ogita-Rump-Oishi), as in the oracle.  (2) Line preconditioner:
 * rows of 256 or more columns take a chunked scan by default (one warp per
 * row, 32 chunks joined by their exact affine maps); with this flag every
 * row takes the oracle's Thomas elimination (one lane per row).  (3) The
 * operator inside the solve: fused multiply-adds by default (9 FP64
 * operations a point instead of 13), the oracle's form with this flag
 * (ftgcr_apply_operator always takes the oracle's form).  The defaults keep
 * the fault decisions of Algorithm 1 and the solution within rounding of the
 * oracle's, but in long, slowly converging solves (the singular mu = 0
 * problem, hundreds of steps) the exit can come some steps earlier or later;
 * with this flag the exit steps are the oracle's.
 * FTGCR_MIXED: FTGCR_ERR_ARG. */
#define FTGCR_FLAG_ORACLE_ORDER 16
/* Every solve of the handle starts from x = 0: x is output only, and its
 * contents on entry are neither read nor checked (host arrays are not copied
 * in).  The results are those of the same solve from a zeroed x (FP64:
 * bitwise); the mixed path also saves the refinement round that would form
 * the first outer residual r_out = R - L(0) = R, taking R for the first inner
 * solve directly.  A host-array solve refused for a non-finite rhs returns
 * x = 0. */
#define FTGCR_FLAG_ZERO_GUESS 32

typedef struct {
  const double* D;   /* [nlat][nlon] cell-centred coefficient (column depth 1 - h), > 0 */
  uint64_t key;      /* serving only: 0, or a caller-chosen identity of D's contents.
                        Passing the same (D, key) pair promises the same contents,
                        so a pooled handle already set up from it is reused without
                        rebuilding its operator and factorisation (the paper's
                        operator is fixed across a model's time steps). */
} ftgcr_coeffs;

/* One single-bit flip: at executed step `step` (1-based, re-executed steps
 * count) XOR bit `bit` of element `index` of vector `vec`.  x, r, p and Ap are
 * hit at the start of the step, before beta is formed; e right after the
 * preconditioner of that step (skipped if the step exits or detects a fault
 * first).  bit is 0..63 of the binary64 pattern (FTGCR_FP64) or 0..31 of the
 * binary32 pattern of the inner vectors (FTGCR_MIXED); in the mixed path
 * `step` counts inner steps across all refinement sweeps. */
typedef struct {
  int64_t step;
  int32_t vec;
  int64_t index;
  int32_t bit;
} ftgcr_fault;

/* One data-loss event, the fault model of Section 3: at executed step `step`,
 * right after the preconditioner (like an e flip), `count` entries of e inside
 * one process block each suffer one bit flip.  The block is `rank` of
 * `nranks` equal contiguous blocks of the row-major array: elements
 * [floor(rank N / nranks), floor((rank + 1) N / nranks)).  Flip i = 1..count
 * takes z = output i of SplitMix64 started at state `seed` (state advanced by
 * 0x9E3779B97F4A7C15 per output, then the generator's published finaliser),
 * element block_start + z mod block_len and bit (z >> 32) mod 64 (FTGCR_FP64)
 * or mod 32 (FTGCR_MIXED).  Two flips of the same bit cancel. */
typedef struct {
  int64_t step;
  int32_t rank;
  int32_t nranks; /* >= 1 */
  int64_t count;  /* >= 0 */
  uint64_t seed;
} ftgcr_loss;

typedef struct {
  const ftgcr_fault* faults; /* host memory, n entries */
  int32_t n;                 /* 0..FTGCR_MAX_FAULTS */
  const ftgcr_loss* losses;  /* host memory, nlosses entries (may be NULL) */
  int32_t nlosses;           /* 0..FTGCR_MAX_LOSSES */
} ftgcr_fault_plan;

#define FTGCR_MAX_LOSSES 16
#define FTGCR_MAX_FAULTS 64
#define FTGCR_MAX_K 16
#define FTGCR_MAX_DETECT 16

typedef struct {
  int64_t steps;           /* executed inner steps (all sweeps) */
  int64_t cycles;          /* completed Krylov cycles (n of Algorithm 1) */
  int64_t restarts;        /* restores of the backup (= detected faults) */
  int64_t faults_injected; /* plan entries that fired */
  int64_t faults_detected;
  int64_t outer;           /* FTGCR_MIXED: refinement sweeps; FTGCR_FP64: 0 */
  int32_t ndetect;         /* entries used in detect_step / detect_ratio */
  int32_t converged;
  int64_t detect_step[FTGCR_MAX_DETECT];   /* step at which each fault was detected */
  double detect_ratio[FTGCR_MAX_DETECT];   /* ||r_new||^2 / ||r_old||^2 at that step */
  double res0;             /* ||L(x0) - R|| */
  double res_final_rec;    /* recurrence residual norm at exit (inner, last sweep) */
  double res_final_true;   /* ||L(x) - R|| of the returned x, FP64 */
  double norm_R;           /* ||R|| */
  int64_t bytes_resident;  /* device bytes held by the handle */
  int64_t bytes_backup;    /* of which the backup [phi, r, p, L(p)]^* (Section 4: 4 arrays) */
  int32_t tiles;           /* row bands used */
  int32_t status;          /* status of the last solve */
  int64_t loss_events;     /* data-loss events that fired */
  int32_t split_rounds;    /* 1: the solve ran split rounds (FTGCR_FLAG_SPLIT_ROUNDS);
                              2: streamed step rounds (FTGCR_FLAG_STREAMED_ROUNDS) */
  int32_t global_factors;  /* 1: FP64 line solve reading its factors from global memory
                              (wide rows: staging them would thin the bands) */
} ftgcr_stats_t;

/* Create a solver for one grid and coefficient field.  Copies D, builds the
 * face coefficients and the line-preconditioner factorisation on the device
 * and allocates every Krylov vector.  k: Krylov cycle length, 1..FTGCR_MAX_K.
 * tol: exit when ||r|| <= tol ||R|| (tol > 0).  Errors: FTGCR_ERR_ARG,
 * FTGCR_ERR_OOM, FTGCR_ERR_CUDA. */
int ftgcr_create(const ftgcr_grid* grid, const ftgcr_coeffs* coeffs, int32_t k, double tol, ftgcr_handle** out);

/* Solve L(x) = rhs (Algorithm 1).  rhs: [N] FP64; x: [N] FP64, in = initial
 * guess, out = solution (host or device memory).  plan: NULL or a fault plan.
 * stream: a cudaStream_t, or NULL for the legacy default stream.  Blocks
 * until done and returns FTGCR_OK, FTGCR_NOT_CONVERGED or an error.  Host
 * arrays are staged and checked on the device: a NaN or an infinity in rhs
 * or x returns FTGCR_ERR_ARG without starting the solve, and leaves x as it
 * was. */
int ftgcr_solve(ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan, void* stream);

/* Same as ftgcr_solve, host arrays included, but only enqueues the work on
 * `stream` and returns: the copies of host arrays into the handle's staging
 * buffers, their finiteness check, the solve and the copy of the solution
 * back into x.  With pinned host arrays the copies run asynchronously, so
 * solves of two handles on two streams overlap one's copies with the other's
 * kernel.  rhs and x must stay valid, and x untouched, until the stream has
 * passed the solve; one solve per handle may be in flight.  ftgcr_stats()
 * (which waits for the stream) then reports its status: FTGCR_ERR_ARG in
 * `status` for a host array holding a NaN or an infinity, x then left as it
 * was.  Returns FTGCR_OK once enqueued, FTGCR_ERR_ARG (null pointer, invalid
 * plan) or FTGCR_ERR_CUDA. */
int ftgcr_solve_host_async(ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan,
                           void* stream);

/* Same as ftgcr_solve but only enqueues the work on `stream` and returns;
 * rhs and x must be device memory.  The status of the solve is read with
 * ftgcr_stats() once the stream has reached the end of the solve.  It
 * allocates nothing and synchronises nothing, so it may be captured into a
 * CUDA graph (stream capture) and the graph replayed. */
int ftgcr_solve_async(ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan, void* stream);

/* Statistics of the last solve of h (synchronises with its stream). */
int ftgcr_stats(ftgcr_handle* h, ftgcr_stats_t* out);

/* Solve n independent problems in ONE persistent launch (all handles of the
 * same precision).  Each solve uses its own handle's tiling, so its result is
 * bitwise the same as when it is solved alone.  rhs[i], x[i] device memory;
 * plans may be NULL.  Enqueues only; read each status with ftgcr_stats().
 * The launch's tables are stream-ordered allocations filled by kernels from
 * their parameters, so the whole batch can be captured into a CUDA graph
 * (after one uncaptured call with the same handles, which configures the
 * kernel) and replayed. */
int ftgcr_solve_batch(ftgcr_handle* const* hs, const double* const* rhs, double* const* x,
                      const ftgcr_fault_plan* const* plans, int32_t n, void* stream);

/* out = L(in), FP64 (device pointers).  The operator of Eq. (1) as built by
 * ftgcr_create. */
int ftgcr_apply_operator(ftgcr_handle* h, const double* in, double* out, void* stream);

/* out = P^-1(in), FP64 (device pointers), with the handle's preconditioner
 * (Algorithm 1, e = P^-1(r)). */
int ftgcr_apply_precond(ftgcr_handle* h, const double* in, double* out, void* stream);

/* Replace the coefficient field of an existing handle: rebuild the face
 * coefficients and the preconditioner factorisation from D (same grid, mu,
 * k and tol), as ftgcr_create does, without reallocating anything.  D:
 * [N] FP64, host or device; a host D is read before the call returns, a
 * device D must stay valid until `stream` has passed this call.  Must not
 * overlap a solve of h.  Errors: FTGCR_ERR_ARG (non-finite or non-positive
 * host D), FTGCR_ERR_CUDA. */
int ftgcr_set_coeffs(ftgcr_handle* h, const ftgcr_coeffs* coeffs, void* stream);

/* Device bytes a handle for this grid would hold (admission control). */
int64_t ftgcr_footprint(const ftgcr_grid* grid, int32_t k);

void ftgcr_destroy(ftgcr_handle* h);
const char* ftgcr_error_string(int status);

/* Tile autotuner.  The paper has no counterpart (it runs one problem per
 * process decomposition).  Row bands and round layout trade halo
 * recomputation against parallelism, and the best trade depends on the grid,
 * the precision and how many solves share a launch.  ftgcr_tune times, for
 * `concurrency` identical solves of this shape in one persistent launch, a
 * set of band counts around the one ftgcr_create picks by itself, each in
 * both round layouts where the mixed path's line preconditioner has two.  It
 * returns the fastest.  Every candidate is a real handle; one whose rows do
 * not fit on chip, or in memory, is skipped.  The problem timed is the
 * caller's operator with a smooth manufactured right-hand side and x0 = 0:
 * one warm launch, then the best of three.  Blocking; allocates (handles,
 * scratch); results are cached per shape for the life of the process (a
 * repeated call returns at once with cached = 1).
 *  - grid: as for ftgcr_create, with tiles = 0 and neither round-layout flag
 *    (the tuner chooses both); coeffs, k, tol as for ftgcr_create.
 *  - concurrency: 1..FTGCR_TUNE_MAX_CONCURRENCY solves per launch.
 *  - Use the result by setting grid.tiles = out->tiles and OR-ing out->flags
 *    into grid.flags.
 *  - Errors: FTGCR_ERR_ARG (arguments, or no candidate fits), FTGCR_ERR_CUDA. */
typedef struct {
  int32_t tiles;          /* chosen row bands */
  int32_t flags;          /* round layout to OR into ftgcr_grid.flags: 0 (FP64, other
                             preconditioners), FTGCR_FLAG_FUSED_ROUNDS, FTGCR_FLAG_SPLIT_ROUNDS or
                             FTGCR_FLAG_STREAMED_ROUNDS */
  double ms;              /* launch time of the chosen layout, ms */
  int32_t default_tiles;  /* the band count ftgcr_create picks by itself */
  double default_ms;      /* its launch time, ms */
  int32_t candidates;     /* layouts timed */
  int32_t cached;         /* 1: returned from the process cache */
} ftgcr_tuning_t;
#define FTGCR_TUNE_MAX_CONCURRENCY 256
int ftgcr_tune(const ftgcr_grid* grid, const ftgcr_coeffs* coeffs, int32_t k, double tol, int32_t concurrency,
               ftgcr_tuning_t* out);

/* No-allocation FP64 solve.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they solve:
 * processes whose device memory belongs entirely to another allocator (a
 * framework's caching pool, a fixed arena reserved at start-up), and code that
 * must not fail with out-of-memory in the middle of a run.  It solves
 * L(x) = rhs like ftgcr_solve with FTGCR_FP64 and the line preconditioner,
 * without a handle, and calls no cudaMalloc, cudaFree or other allocating
 * routine: every Krylov vector, coefficient, factor and bookkeeping record
 * lives in one static device array of FTGCR_NOALLOC_SCRATCH_BYTES that every
 * GPU loading the library holds until the process exits.
 *  - Limits: nlon * nlat <= FTGCR_NOALLOC_MAX_POINTS, k <= FTGCR_NOALLOC_MAX_K;
 *    larger sizes return FTGCR_ERR_ARG.
 *  - D, rhs, x: device pointers (x: initial guess in, solution out); stats
 *    may be NULL.  Returns like ftgcr_solve.
 *  - The call is blocking: it copies the grid geometry and the solve record
 *    from host (stack) memory to the device, copies the result record back,
 *    and synchronises the stream before it returns.  It is therefore not for
 *    use while a stream is being captured into a CUDA graph
 *    (ftgcr_solve_async is the capturable solve).
 *  - It does not raise the per-thread stack limit (that may allocate): the
 *    current cudaLimitStackSize must cover the solve kernel's frame plus
 *    256 bytes, the margin ftgcr_create keeps, or the call returns
 *    FTGCR_ERR_ARG.  The CUDA default limit covers the FP64 kernels; an
 *    earlier ftgcr_create or the caller may also have raised it.
 *  - The first call on a device looks up the array's device address (set-up).
 *  - All calls share the array, which keeps the last call's contents; each
 *    call clears the part it uses before it starts, so a result does not
 *    depend on earlier calls.  Calls that overlap on the GPU (other threads,
 *    other streams) race and must be serialised by the caller. */
#define FTGCR_NOALLOC_MAX_POINTS 16384
#define FTGCR_NOALLOC_MAX_K 4
#define FTGCR_NOALLOC_SCRATCH_BYTES (6 * 1024 * 1024)
int ftgcr_solve_noalloc(const ftgcr_grid* grid, const double* D, int32_t k, double tol, const double* rhs, double* x,
                        ftgcr_stats_t* stats, void* stream);

/* ---- serving: continuous batching of independent solves ----
 * The paper solves one elliptic problem per model time step (Section 2); a
 * server runs many such requests at once.  It owns a scheduler thread, a
 * preparation thread, CUDA streams for launches, copies and set-up, a pool of
 * solver handles and two tables of max_slots solve slots (one per precision).
 * A queued request first gets a handle (first come, first served, within the
 * budget); a handle that must be created or rebuilt from the request's
 * coefficients is prepared on the preparation thread, so set-up never holds
 * up the running solves.  Each epoch the scheduler admits ready requests, in
 * submission order, while a slot of their precision is free, runs every
 * running solve for at most epoch_rounds rounds of one persistent launch, and
 * hands back the solves that finished.  Unfinished solves resume in the next
 * epoch beside the newly admitted ones.  Every result, statistics included,
 * is bitwise the result of the same request solved alone with ftgcr_solve.
 *  - Memory: a request is charged ftgcr_footprint(grid, k) while its handle is
 *    held; idle handles are pooled by shape (grid, k, tol).  A request takes an
 *    idle handle already set up from the same (D, key) as is; otherwise a new
 *    handle is made while the budget allows (a keyless request rebuilds an
 *    idle handle of its shape first), then an idle handle of the shape is
 *    rebuilt, then idle handles are evicted least recently used first.
 *    budget_bytes = 0 means half of the device memory free at creation.
 *  - Pointers: D, rhs and x may be host or device memory and must stay valid,
 *    and x untouched by the caller, until poll/wait reports the result.  Host
 *    rhs and x are staged (pinned host memory is copied asynchronously) and
 *    checked for finite values on the device: a request holding a NaN or an
 *    infinity does not start and completes with FTGCR_ERR_ARG, x unchanged.
 *  - Thread safety: submit, poll, wait and info may be called from any
 *    thread; destroy must not overlap any other call on the same server. */
typedef struct ftgcr_server ftgcr_server;
typedef struct {
  int64_t submitted, completed;
  int64_t queued;       /* waiting for a handle, in preparation or for a slot */
  int64_t running;
  int64_t epochs;       /* persistent launches made */
  int64_t handles;      /* handles held (running and pooled) */
  int64_t bytes_in_use; /* their footprint */
  int64_t budget_bytes;
} ftgcr_server_info_t;

/* Start a server on the current device.  max_slots: 1..1024 solves of each
 * precision running at once; epoch_rounds >= 1 rounds per launch (an inner
 * step takes two).  Errors: FTGCR_ERR_ARG, FTGCR_ERR_OOM, FTGCR_ERR_CUDA. */
int ftgcr_server_create(int64_t budget_bytes, int32_t max_slots, int32_t epoch_rounds, ftgcr_server** out);

/* Queue one solve of L(x) = rhs for the grid and coefficients given (as
 * ftgcr_create + ftgcr_solve would).  plan: NULL or a fault plan (copied).
 * *ticket identifies the request.  Errors: FTGCR_ERR_ARG (bad grid, k, tol,
 * pointer or plan), FTGCR_ERR_BUDGET (footprint above the whole budget),
 * FTGCR_ERR_STATE (server stopping). */
int ftgcr_server_submit(ftgcr_server* srv, const ftgcr_grid* grid, const ftgcr_coeffs* coeffs, int32_t k, double tol,
                        const double* rhs, double* x, const ftgcr_fault_plan* plan, int64_t* ticket);

/* FTGCR_PENDING while the request runs; once it has finished, its status
 * (as ftgcr_solve returns it) with *stats filled (stats may be NULL), after
 * which the ticket is released.  FTGCR_ERR_ARG for an unknown ticket. */
int ftgcr_server_poll(ftgcr_server* srv, int64_t ticket, ftgcr_stats_t* stats);

/* Like poll, but blocks until the request finishes or timeout_s seconds pass
 * (timeout_s < 0: no limit); FTGCR_PENDING on timeout. */
int ftgcr_server_wait(ftgcr_server* srv, int64_t ticket, double timeout_s, ftgcr_stats_t* stats);

/* Completion queue: the earliest-finished request not yet collected, with its
 * ticket in *ticket, its status returned and *stats filled, as poll does;
 * FTGCR_PENDING if none finishes within timeout_s seconds (timeout_s < 0: no
 * limit, but FTGCR_ERR_STATE when no request is outstanding at all). */
int ftgcr_server_next(ftgcr_server* srv, double timeout_s, int64_t* ticket, ftgcr_stats_t* stats);

int ftgcr_server_info(ftgcr_server* srv, ftgcr_server_info_t* out);

/* Admission limit: at most max_points grid points (nlon * nlat summed over
 * the running solves) per precision at once; 0 (the default) means no limit.
 * Every running solve advances one round per round of the shared launch, and
 * a round's time grows with the points in it, so the limit trades throughput
 * for shorter rounds: the request that would cross it waits, in submission
 * order, and so do the requests behind it; a request alone in its precision
 * always runs.  Takes effect from the next epoch.  Errors: FTGCR_ERR_ARG. */
int ftgcr_server_set_max_points(ftgcr_server* srv, int64_t max_points);

/* Stop: queued requests end with FTGCR_ERR_STATE, running ones finish; then
 * every handle and buffer is freed. */
int ftgcr_server_destroy(ftgcr_server* srv);

/* Measurement probe, off every solve path: the device's FP64 fused
 * multiply-add rate in TFLOP/s (2 flops per FMA), from one launch of
 * independent FMA chains filling every SM, timed with CUDA events on
 * `stream` (NULL: the default stream).  It is the ceiling of the FP64 path's
 * arithmetic: its row-solve chains and compensated dot products run on the
 * FP64 pipe.  iters: FMAs per chain, 1 .. 2^24 (about 4096 takes a few ms on
 * GB300).  Blocks the host until the launch ends.  Errors: FTGCR_ERR_ARG (iters
 * out of range or tflops NULL), FTGCR_ERR_OOM, FTGCR_ERR_CUDA; *tflops is 0
 * on error. */
int ftgcr_fp64_fma_rate(int32_t iters, double* tflops, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FTGCR_H */
