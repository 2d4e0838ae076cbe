/*
 * aao.h -- C ABI of the GB300 all-at-once wave solver (libaao.so).
 *
 * The library solves the symmetrised all-at-once system of the implicit
 * leap-frog discretisation of the wave equation
 *
 *     u_tt = c^2 Lap u + f   on (0,1)^d x (0,T],  u = 0 on the boundary,
 *     u(0) = psi0, u_t(0) = psi1                      (paper, eq. (1.1))
 *
 * by preconditioned MINRES on  Y T u = Y f  (eqs. (main_matrix), (symmetricform))
 * with the absolute-value block alpha-circulant preconditioner
 * P_alpha = (C_alpha^{1/2})^T C_alpha^{1/2}  (def. (matrix_P), eq. (precsys)).
 *
 * Conventions shared by every entry point
 *   - grid: d in {1,2,3}; N interior points per axis, the same on every axis;
 *     h = 1/(N+1); m = N^d spatial unknowns in lexicographic order, x fastest.
 *   - time: nt = n time levels u^(1..n), tau = T/n (the caller passes tau).
 *   - vectors: FP64, time-major, index (rhs, i, s) -> (rhs*n + i)*m + s with
 *     i = 0..n-1 standing for u^(i+1).  A batch of nrhs vectors is contiguous.
 *   - pointers are DEVICE pointers unless an entry point says otherwise; they
 *     are owned by the caller and must stay valid until the stream reaches the
 *     end of the call.  Alignment: 8 bytes.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are stream-ordered and asynchronous except where stated.
 *   - errors: every call returns an aao_status; nothing is thrown across the
 *     ABI.  aao_last_error() gives a thread-local text for the last failure.
 *   - a handle may be used from one host thread at a time.
 */
#ifndef AAO_H_
#define AAO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum aao_status {
  AAO_OK = 0,
  AAO_EINVAL = 1,        /* bad argument (null pointer, alpha outside (0,1], tau <= 0, ...) */
  AAO_EUNSUPPORTED = 2,  /* size outside what the kernels implement (see aao_create) */
  AAO_ENOMEM = 3,        /* device allocation failed, or a request exceeds a budget */
  AAO_ECUDA = 4,         /* a CUDA runtime call failed; aao_last_error() has the text */
  AAO_ENOTCONV = 5,      /* MINRES reached maxit before the residual tolerance */
  AAO_EBREAKDOWN = 6,    /* MINRES breakdown: <z, v> < 0 (preconditioner not SPD in floating point) */
  AAO_ESINGULAR = 7,     /* preconditioner singular: min |Sigma| below the threshold (alpha = 1 only) */
  AAO_EBUSY = 8,         /* serving: no free slot */
  AAO_EPENDING = 9,      /* serving: request not finished yet */
  AAO_ETIMEOUT = 10      /* a bounded wait ran out */
} aao_status;

/* Spatial grid: Omega = (0,1)^dim, N interior points per axis (equal spacing on
 * every axis, as in the paper's Section 3), wave speed squared c2 (1 in the paper;
 * L = I - (c2 tau^2 / 2) Delta_h, i.e. the mean-coefficient form of eq.
 * (mean-coefftsmat) with a-bar = c2). */
typedef struct aao_grid {
  int dim;
  int N;
  double c2;
} aao_grid;

/* Time discretisation: the implicit leap-frog scheme of Section 1 (the only one). */
typedef enum aao_scheme { AAO_SCHEME_IMPLICIT_LEAPFROG = 0 } aao_scheme;

/* Precision of the preconditioner application. */
typedef enum aao_precision {
  AAO_PREC_FP64 = 0,     /* everything in FP64 */
  AAO_PREC_FP32_IR = 1,  /* P_alpha^{-1} in FP32/complex64; operator, MINRES recurrences,
                            residuals and an outer iterative refinement in FP64; the DSTs
                            of b and x (and aao_apply_dst) in double-float (see below) */
  AAO_PREC_F32X2 = 2     /* P_alpha^{-1} (DSTs and time part) and the DSTs of the solve in
                            double-float arithmetic (pairs of FP32 numbers, ~47 significant
                            bits, on the FP32 pipes) on FP64 vectors; operator, recurrences and
                            residuals in FP64; no refinement loop (not a mode of the paper: a
                            GB300 design choice, whose FP64 pipe issues 64 times fewer
                            operations per clock than its FP32 pipes) */
} aao_precision;

typedef struct aao_opts {
  int precision;         /* aao_precision, default AAO_PREC_FP64 */
  int nrhs_max;          /* largest batch passed to any call; workspace is sized for it (default 1) */
  int variable_coefficient; /* != 0: reserve room for a coefficient set by aao_set_coefficient */
  int graph;             /* != 0: aao_minres_solve captures its iteration loop once per (batch
                            size, initial-guess use) into a CUDA graph whose device-side WHILE
                            node runs the iterations without host round trips (bounded by
                            maxit); tolerance and maxit are written to device memory before
                            each launch, so they may change between calls without a new
                            capture; when kernel timing is enabled the host-driven loop is used */
  int host_staging;      /* != 0: aao_create also reserves the device buffers, copy stream and
                            events of aao_solve_host (for nrhs_max right-hand sides), so that no
                            later call allocates; 0: the first aao_solve_host reserves them */
  int reserved[3];       /* must be zero */
} aao_opts;

typedef struct aao_solve_info {
  int iters;             /* MINRES iterations (summed over refinement steps in FP32_IR mode) */
  int status;            /* aao_status of this right-hand side */
  double relres_true;    /* ||b - Y T x||_2 / ||b||_2, recomputed explicitly */
  double relres_est;     /* MINRES recurrence estimate ||r||_{P^-1} / ||r_0||_{P^-1} */
  int ir_steps;          /* outer refinement steps (FP32_IR mode), else 0 */
  int reserved;
} aao_solve_info;

typedef struct aao_handle aao_handle;

/* Create a solver for one (grid, nt, tau, alpha) and allocate all its device
 * memory (tables + workspace); this is the only allocating call besides the
 * serving API and, for a handle created without opts.host_staging, the first
 * aao_solve_host.  Builds, on the device, the spectral factors
 * Sigma_{k,j}^{-1/2} = (Lambda_j lambda_{1,k} + lambda_{2,k})^{-1/2} with the
 * principal branch (eqs. (calphaprediagform), (calphasqrtdiagform); Section 2.3).
 *   grid  : host pointer; dim in {1,2,3}; N+1 a power of two, 64 <= N+1 <= 512
 *           (so N in {63,127,255,511}); c2 > 0.
 *   nt    : number of time levels n; a power of two, 64 <= nt <= 1024.
 *   tau   : time step (> 0), normally T/nt.
 *   alpha : in (0, 1]; alpha = 1 gives the ABC preconditioner |C_1| (Remark
 *           p1badpermformremark) and returns AAO_ESINGULAR if some |Sigma| is
 *           below 1e-12 * max|Sigma| (Remark c1badperformremark).
 *   scheme: AAO_SCHEME_IMPLICIT_LEAPFROG.
 *   opts  : host pointer or NULL for defaults.
 *   out   : receives the handle (host pointer).
 * The tables are built on a non-blocking stream owned by the handle, and the call
 * returns once that stream is done: it does not wait for work that other streams
 * have in flight on the device.
 * Tuning overrides (environment, read here; for measurements and tests):
 *   AAO_TIME_VARIANT="v64[,v32[,vff]]" sets the time-kernel variant per precision
 *   (the numbering of aao_autotune; a missing entry repeats the previous one), and
 *   AAO_DST_VARIANT="0..8" the DST variant (bit 0: radix-16-first stage plan, bit 1:
 *   batched loads, bit 2: interleaved padded shared-memory layout; 8: the one-warp
 *   small-problem tile), AAO_SMALL_TILES=0 keeps the
 *   standard tiles for a small problem (by default a problem whose standard tiles
 *   would occupy fewer than a quarter of the SMs gets the one-warp time (variant 30)
 *   and DST tiles, operator runs of 4 time levels and the small w/x update shape;
 *   served handles always keep the standard tiles), and AAO_FUSED_SCALARS=1 runs the MINRES scalar steps in the tails
 *   of the kernels that produce their partial sums (five launches per iteration instead
 *   of eight, and no separate loop-condition launch in a graph trip).  Every variant
 *   computes the same values (bit for bit, for the fused scalar steps).
 * Errors: AAO_EINVAL, AAO_EUNSUPPORTED, AAO_ENOMEM, AAO_ECUDA, AAO_ESINGULAR. */
aao_status aao_create(const aao_grid* grid, int nt, double tau, double alpha,
                      aao_scheme scheme, const aao_opts* opts, aao_handle** out);

/* Variable coefficient u_tt = div(a grad u) + f (Section 3, eq. (var coeff wave)):
 * from this call on, the operator (aao_apply_op, aao_build_rhs, aao_residual_norm and
 * the solves) uses L_a = I - (tau^2/2) Delta_{a,h} with the conservative central
 * difference (Delta_{a,h} w)_i = sum_axes [a_{i+1/2}(w_{i+1} - w_i) - a_{i-1/2}(w_i - w_{i-1})]/h^2
 * (eq. (tssystemvarwaveeq); the second right-hand-side block uses L_a psi0), while
 * the preconditioner keeps the constant coefficient grid->c2 given to aao_create
 * (the mean-coefficient preconditioner of eq. (mean-coefftsmat): pass c2 = mean of a
 * on the grid).  MINRES then runs in the physical basis.
 *   a_face : device array, the d face arrays one after the other; the array of axis
 *            ax (0 = x) has N+1 entries along ax (face f at coordinate (f + 1/2) h,
 *            f = 0..N) and N along the others, lexicographic with x fastest; total
 *            d (N+1) N^(d-1) doubles.  Copied (stream-ordered) into the handle.
 * The handle must have been created with opts.variable_coefficient != 0.
 * Errors: AAO_EINVAL, AAO_ECUDA. */
aao_status aao_set_coefficient(aao_handle* h, const double* a_face, void* stream);

/* Free the handle and all its device memory (synchronises its device). */
aao_status aao_destroy(aao_handle* h);

/* Bytes of device memory held by the handle (tables + workspace). */
size_t aao_workspace_bytes(const aao_handle* h);

/* Build b = Y f from the data of eq. (main_matrix):
 *   f    : nrhs x n x m, f[k] = f(G_h, k tau), k = 0..n-1 (source samples);
 *   psi0 : nrhs x m, psi1: nrhs x m (initial value and velocity);
 *   b    : nrhs x n x m output, the time-reversed right-hand side
 *          tau^2 [f^0/2 + psi1/tau + psi0/tau^2; f^1 - L psi0/tau^2; f^2; ...; f^(n-1)].
 * Device pointers; b must not alias the inputs.  Errors: AAO_EINVAL, AAO_ECUDA. */
aao_status aao_build_rhs(aao_handle* h, const double* f, const double* psi0,
                         const double* psi1, double* b, int nrhs, void* stream);

/* y = Y T x (eq. (main_system)): (T x)_i = L x_i - 2 x_{i-1} + L x_{i-2} with
 * x_{-1} = x_{-2} = 0, L = I - (c2 tau^2/2) Delta_h the (2d+1)-point Dirichlet
 * stencil, and Y reversing the time levels (Section 2.3, first paragraph).
 * x, y: nrhs x n x m device vectors, must not alias.  Errors: AAO_EINVAL, AAO_ECUDA. */
aao_status aao_apply_op(aao_handle* h, const double* x, double* y, int nrhs, void* stream);

/* z = P_alpha^{-1} r = C_alpha^{-1/2} (C_alpha^{-1/2})^T r by Section 2.3's
 * three-step procedure done twice: a DST along each spatial axis, per spatial
 * mode the time pipeline D^{-1} -> FFT -> x Sigma^{-1/2} -> iFFT -> D^2 ->
 * FFT -> x conj(Sigma^{-1/2}) -> iFFT -> D^{-1}, then the DSTs again.
 * r, z: nrhs x n x m device vectors; z may equal r (in place).  Uses the
 * handle's precision (in FP32 mode through an FP32 buffer of nrhs_max x n x m floats
 * that aao_create reserves).  Errors: AAO_EINVAL, AAO_ECUDA. */
aao_status aao_apply_prec(aao_handle* h, const double* r, double* z, int nrhs, void* stream);

/* y = (I_n (x) U) x with U = S (x) ... (x) S the orthonormal multi-dimensional
 * DST-I (Section 2.3: on a uniform grid the eigenvector matrix U of L is the
 * DST); U = U^T = U^{-1}.  This is the spatial part of P_alpha^{-1}, exposed on
 * its own.  x, y: nrhs x n x m FP64 vectors, may be equal; FP64 arithmetic, or
 * double-float for AAO_PREC_F32X2 and AAO_PREC_FP32_IR handles.  Errors: AAO_EINVAL,
 * AAO_ECUDA. */
aao_status aao_apply_dst(aao_handle* h, const double* x, double* y, int nrhs, void* stream);

/* The time part of P_alpha^{-1} on DST coefficients: for every spatial mode j
 * the n x n map D^{-1} F^* G_j F D^2 F G_j F^* D^{-1} (G_j = diag of
 * Sigma_{k,j}^{-1/2}; Section 2.3 with U factored out), so that
 * apply_prec = apply_dst o apply_time o apply_dst.  x, y may be equal.  FP64
 * vectors; the arithmetic is the handle's precision (FP32/complex64 for
 * AAO_PREC_FP32_IR, converted on load and store).  Errors: AAO_EINVAL, AAO_ECUDA. */
aao_status aao_apply_time(aao_handle* h, const double* x, double* y, int nrhs, void* stream);

/* Preconditioned MINRES on Y T x = b with P_alpha (eq. (precsys); Section 3:
 * MINRES, relative-residual stopping).  Stops for each right-hand side at the
 * first iteration whose TRUE relative residual ||b - Y T x||_2/||b||_2 <= rtol
 * (recomputed every iteration), or at maxit.
 *   b      : nrhs x n x m device input (unchanged).
 *   x      : nrhs x n x m device in/out: the initial guess if use_x0 != 0
 *            (else ignored and zero is used, as in the paper), the solution on return.
 *   info   : host array of nrhs records (may be NULL).
 * Blocks the calling thread until the solve finishes (it reads a small status
 * block every iteration).  Returns AAO_OK if every right-hand side converged,
 * else the first failing status (AAO_ENOTCONV, AAO_EBREAKDOWN), with info
 * filled in either case.  Errors also: AAO_EINVAL, AAO_ECUDA. */
aao_status aao_minres_solve(aao_handle* h, const double* b, double* x, int use_x0, int nrhs,
                            double rtol, int maxit, aao_solve_info* info, void* stream);

/* relres[r] = ||b_r - Y T x_r||_2 / ||b_r||_2 for every right-hand side r: the
 * true relative residual that aao_minres_solve stops on (Section 3: MINRES with
 * a relative-residual stopping rule; Y T as in aao_apply_op).  If ||b_r|| = 0
 * the absolute residual norm is returned.
 *   b, x   : nrhs x n x m device vectors (inputs, unchanged).
 *   relres : device array of nrhs doubles (output), written stream-ordered.
 * Uses the handle's reduction workspace, so calls on one handle must not
 * overlap.  Errors: AAO_EINVAL (null pointer, nrhs outside [1, nrhs_max]), AAO_ECUDA. */
aao_status aao_residual_norm(aao_handle* h, const double* b, const double* x, double* relres,
                             int nrhs, void* stream);

/* Allocation-free variant of aao_residual_norm.  The paper has no counterpart:
 * it is a library facility for callers that cannot allocate device memory at the
 * point where they need a residual check -- e.g. plugin code inside a host
 * framework whose pool allocator owns all device memory and forbids outside
 * allocations, or a latency-critical loop where the implicit synchronisation of
 * cudaMalloc/cudaFree is not acceptable.  It takes no handle (creating one
 * allocates) and calls no cudaMalloc, cudaFree or other allocating routine.
 *   grid, nt, tau : as for aao_create (host pointer for grid); any N >= 1, nt >= 1.
 *   b, x          : nrhs x n x m device vectors (inputs); relres: nrhs device doubles (output).
 *   nrhs          : 1..64.  Larger values return AAO_EINVAL: the scratch is a static
 *                   device array of 32768 doubles (256 KiB, 512 partial sums per
 *                   right-hand side).
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current.  Under CUDA's lazy module loading
 * (the default) that lookup also loads the array and its kernels onto the device, a
 * one-time driver allocation of about 256 KiB plus code that stays until the process
 * exits: make the first call at initialisation time, before any stream capture and
 * before the caller's allocator takes the device's memory; later calls allocate
 * nothing.  The looked-up address does not survive cudaDeviceReset: after a reset
 * the entry point must not be called again.  All calls share the array and it keeps the last call's
 * partial sums (each call rewrites every slot it reads, so nothing needs
 * clearing); calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race on it and must be serialised by the caller.
 * Errors: AAO_EINVAL, AAO_ECUDA; text in aao_noalloc_last_error(). */
aao_status aao_residual_norm_noalloc(const aao_grid* grid, int nt, double tau, const double* b,
                                     const double* x, double* relres, int nrhs, void* stream);

/* Thread-local text of the last aao_residual_norm_noalloc failure ("" if none). */
const char* aao_noalloc_last_error(void);

/* End-to-end solve from HOST buffers: copies f, psi0, psi1 (host, any memory;
 * pinned for speed) to the device, builds b (aao_build_rhs), runs
 * aao_minres_solve from a zero guess, and copies u (host, nrhs x n x m) back.
 * For constant-coefficient FP64 and double-float handles the copies run on a
 * second stream in chunks of 32 time levels, overlapping the right-hand side and
 * the DSTs (each level of those depends on its own f level only; the result is
 * bit for bit the device-buffer solve).  The device copies of f, b, x, the copy
 * stream and its events are reserved by aao_create if opts.host_staging was set,
 * else by the first call (which then allocates).  Blocks until u is on the host.
 * Errors as aao_minres_solve, and AAO_ENOMEM. */
aao_status aao_solve_host(aao_handle* h, const double* f, const double* psi0, const double* psi1,
                          double* u, int nrhs, double rtol, int maxit,
                          aao_solve_info* info, void* stream);

/* ---------------------------------------------------------------------------
 * Serving: a request loop that admits solves of mixed sizes, wave speeds, alpha
 * and tolerances onto one GPU under an HBM budget (continuous admission: requests
 * that arrive while others run are started as slots and memory free up; their work
 * runs concurrently on the device).  Not part of the paper: a runtime around its
 * method.  Each request is a solve of eq. (precsys) as aao_minres_solve does it in
 * the request's precision (FP64 or double-float; zero initial guess, true relative
 * residual <= rtol); the Krylov state stays on
 * the device for the whole solve, whose iterations run in grouped launches with the
 * other requests of its size class (one CUDA stream per class, the smaller classes at
 * the higher stream priorities); a request never shares buffers with another and its
 * blocks run the code and decomposition of its solo solve, so its result does not
 * depend on what else is running (bit for bit the solo solve of a handle created with
 * AAO_SMALL_TILES=0: served handles keep the standard tiles).
 * --------------------------------------------------------------------------- */
typedef struct aao_server aao_server;

typedef struct aao_request {
  int dim, N, nt;        /* shape, as for aao_create (N+1 and nt powers of two in range) */
  double tau, alpha, c2; /* time step, alpha in (0,1], wave speed squared */
  double rtol;           /* true relative residual tolerance */
  int maxit;
  const double* f;       /* device, n x m source samples (as for aao_build_rhs) */
  const double* psi0;    /* device, m */
  const double* psi1;    /* device, m */
  double* x;             /* device, n x m solution output (written by the server) */
  int precision;         /* AAO_PREC_FP64 (0, the default of a zeroed request) or
                            AAO_PREC_F32X2; the refinement mode is not served */
} aao_request;

typedef struct aao_serve_result {
  aao_solve_info info;   /* iterations, status, residuals of this request */
  double t_submit;       /* seconds since aao_serve_create: submitted */
  double t_start;        /* admitted and enqueued on the GPU */
  double t_done;         /* completion observed by the server */
  uint64_t ticket;
} aao_serve_result;

typedef struct aao_serve_stats {
  uint64_t submitted, admitted, completed, failed, handles_created, evictions;
  uint64_t pool_bytes, peak_pool_bytes, budget;
  int in_flight, pending;
  uint64_t rounds;           /* grouped MINRES iterations run (one per size class and step) */
  uint64_t round_problems;   /* requests summed over those rounds (/ rounds = mean group size) */
  uint64_t grouped_launches; /* kernel launches of those rounds */
} aao_serve_stats;

/* Start a server on the current device.  hbm_budget_bytes bounds the device memory
 * of its handle pool (workspace + tables + right-hand-side buffers); max_slots (1..64)
 * bounds the solves in flight.  Allocates nothing until requests arrive.
 * Errors: AAO_EINVAL, AAO_ECUDA. */
aao_status aao_serve_create(size_t hbm_budget_bytes, int max_slots, aao_server** out);

/* Queue a request (host pointer r, copied; the device buffers it names must stay
 * valid and unchanged until the request completes).  Returns a ticket.  Never blocks
 * on the GPU.  Errors: AAO_EINVAL, AAO_EUNSUPPORTED (size), AAO_EBUSY (shutting down).
 * A request whose handle can never fit the budget completes with AAO_ENOMEM. */
aao_status aao_serve_submit(aao_server* s, const aao_request* r, uint64_t* ticket);

/* Non-blocking: AAO_EPENDING until the request finished, then its status (AAO_OK,
 * AAO_ENOTCONV, ...) with *out filled; a finished ticket can be read once.
 * AAO_EINVAL for an unknown ticket. */
aao_status aao_serve_poll(aao_server* s, uint64_t ticket, aao_serve_result* out);

/* Like aao_serve_poll but waits up to timeout_s seconds; AAO_ETIMEOUT if still pending. */
aao_status aao_serve_wait(aao_server* s, uint64_t ticket, double timeout_s, aao_serve_result* out);

/* Counters (host pointer). */
aao_status aao_serve_stats_get(aao_server* s, aao_serve_stats* out);

/* Finish every queued and running request, then free all handles and streams. */
aao_status aao_serve_destroy(aao_server* s);

/* Thread-local text of the last serving failure in this thread. */
const char* aao_serve_last_error(void);

/* Autotuner: pick, for this handle's shape and precision, the fastest variant of the
 * time-pipeline kernel (FFT stage plan: radix-4 or radix-16 first; tile: 4096/n or
 * 2048/n mode pairs per CTA; shared-memory layout: sequence-major or interleaved and
 * padded, the latter with or without a staged slice of the spectral table; and, for
 * the FP32 and double-float pipelines on FP64 vectors, loads batched ahead of their
 * conversion, bulk-copy staging of the tile or integer conversions (of the loads, the
 * stores or both), and, in FP32, the spectral table read from memory or computed on
 * the fly) and of the DST
 * kernel (radix-4 or radix-16 stage plan, with or without batched loads, sequence-major
 * or interleaved shared-memory layout, or the small-problem tile) by timing
 * each on the handle's workspace with CUDA events (the work of the kernels is
 * the same in every variant; only speed differs).  The default variant is kept unless
 * another is more than 1 % faster, so near-ties give the same choice on every run.
 * tune_file (host string, may be
 * NULL): a text file of cached choices, one line "dim N nt precision time dst"; a
 * matching line is applied without measuring, otherwise the measured choice is
 * appended.  chosen (host, may be NULL): receives {time variant, DST variant}.
 * Synchronous; must not overlap other calls on the handle.  Errors: AAO_EINVAL,
 * AAO_ECUDA. */
aao_status aao_autotune(aao_handle* h, const char* tune_file, int* chosen);

/* Number of kernel launches this handle has issued since creation (statistics). */
uint64_t aao_launch_count(const aao_handle* h);

/* Arithmetic-rate probe (statistics for rooflines, not part of the method): times, with
 * CUDA events on a private stream, a kernel of independent fused multiply-add chains on
 * every SM (8 blocks of 256 threads per SM, 8 chains per thread, `iters` steps per
 * chain; best of 3 after a warm-up) and returns the rate in TFLOP/s (2 flops per FMA)
 * and the kernel time.  precision: AAO_PREC_FP64 (DFMA) or AAO_PREC_FP32_IR (FFMA).
 * Synchronous; allocates one scalar.  Errors: AAO_EINVAL, AAO_ENOMEM, AAO_ECUDA. */
aao_status aao_alu_peak(int precision, int iters, double* tflops, double* ms);

/* Kernels that stage data with bulk asynchronous copies wait on an mbarrier with a
 * bounded number of polls; a wait that runs out is counted here (process-wide, current
 * device) and its tile is abandoned.  0 in a healthy run; 0xFFFFFFFF if the counter
 * cannot be read.  Statistics, not part of the method. */
unsigned int aao_wait_timeouts(void);

/* Per-kernel timing (statistics, not part of the method).  While enabled, every
 * kernel the handle launches is bracketed by two CUDA events recorded on the
 * stream it is launched on; aao_profile_read synchronises on those events and
 * returns, per kernel class, the launch count and the summed event time. */
typedef struct aao_kernel_stat {
  char name[32];         /* kernel class, e.g. "dst_x_f64", "time_f64", "yt_dot" */
  uint64_t launches;
  double total_ms;
} aao_kernel_stat;

/* on != 0: clear the records and start recording; on == 0: stop recording
 * (records are kept until the next enable).  Errors: AAO_EINVAL. */
aao_status aao_profile_enable(aao_handle* h, int on);

/* Fill out[0..max) with the classes seen since the last enable (host array) and
 * return how many there are (may exceed max), or -1 on error.  Blocks until
 * every recorded event has completed. */
int aao_profile_read(aao_handle* h, aao_kernel_stat* out, int max);

/* Text of a status code (static storage). */
const char* aao_status_str(aao_status s);

/* Thread-local text of the last failure in this thread ("" if none). */
const char* aao_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* AAO_H_ */
