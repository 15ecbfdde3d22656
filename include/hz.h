/*
 * hz.h - C ABI of the GB300 shifted-Laplacian multigrid Helmholtz solver.
 *
 * Solves the 2-D Helmholtz problem  Delta u + k(x)^2 u = f  on the unit square with
 * first-order Sommerfeld boundaries  du/dn - i k u = 0  (arXiv 1312.2880, Sec. 1, Eq. 1),
 * discretised by the 5-point stencil L^h (Eq. 2), with Bi-CGSTAB (Sec. 6) right-
 * preconditioned by a multigrid V-cycle whose levels relax with L^H or with the shifted
 * operator M^H = L^H + i k^2 beta (Eq. 3) as the HLM-V / SL-V / HYB-V variants prescribe
 * (Sec. 5): red-black Gauss-Seidel on most scales, 5-colour Kaczmarz (Gauss-Seidel on the
 * normal equations, Sec. 4-5) on the kH ~ 1.25 scale, full weighting, bilinear
 * interpolation and a dense solve on the coarsest grid.
 *
 * Conventions shared by every entry point
 *  - Grid: (n+1) x (n+1) vertex nodes of [0,1]^2, h = 1/n, boundary nodes are unknowns.
 *    Node (i, j) sits at (i h, j h); arrays are row-major with i (x) fastest:
 *    element (i, j) of a level-l array is at index j*(n_l+1) + i, n_l = n / 2^l.
 *  - Complex vectors are interleaved complex128 (re, im doubles), i.e. the layout of
 *    C99 double complex, numpy complex128 and torch.complex128.
 *  - Units are the paper's: rows carry the 1/h^2 factor; u and x are unscaled.
 *  - Pointers documented "device" must be device memory of the current CUDA device that is
 *    valid on the problem's stream; "host" pointers are ordinary host memory. The caller owns
 *    every array it passes; the library never keeps a caller pointer after a call returns.
 *  - Every call is asynchronous on the problem's stream unless it says it synchronises.
 *    Calls that return results to host memory synchronise that stream.
 *  - Errors are returned as hz_status; the message of the last failure on a problem is
 *    available from hz_last_error. No call aborts, exits or traps on the device.
 *  - A problem is not thread-safe: one host thread and one stream per problem.
 */
#ifndef HZ_H
#define HZ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hz_problem hz_problem; /* opaque; created by hz_create_problem, freed by hz_destroy */

typedef enum {
  HZ_OK = 0,
  HZ_EINVAL = 1,      /* bad argument (size, pointer, option); nothing was launched */
  HZ_ENOMEM = 2,      /* arena too small or device allocation refused */
  HZ_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed; see hz_last_error */
  HZ_ENOTSETUP = 4,   /* hz_setup_hierarchy has not been called */
  HZ_EBREAKDOWN = 5,  /* Bi-CGSTAB breakdown (rho, <r^,v> or omega exactly zero) */
  HZ_EMAXIT = 6,      /* maxit iterations without reaching tol; x holds the last iterate */
  HZ_ENONFINITE = 7,  /* a NaN or Inf appeared in the Krylov scalars (e.g. non-finite input) */
  HZ_ETIMEOUT = 8     /* a bounded device-side wait ran out */
} hz_status;

typedef enum { HZ_BC_SOMMERFELD1 = 0 } hz_bc; /* first-order Sommerfeld rows by ghost elimination */

/* V-cycle variants of Sec. 5. HZ_VAR_SL_PLAIN: M^H with Gauss-Seidel on every level. */
typedef enum { HZ_VAR_HYB = 0, HZ_VAR_SL = 1, HZ_VAR_HLM = 2, HZ_VAR_SL_PLAIN = 3 } hz_variant;

/* Arithmetic of the V-cycle. The Bi-CGSTAB vectors, recurrences, dot products and the
 * true-residual check are always complex FP64. */
typedef enum { HZ_PREC_FP64 = 0, HZ_PREC_FP32 = 1 } hz_prec;

typedef enum { HZ_OP_L = 0, HZ_OP_M = 1 } hz_op;
typedef enum { HZ_SMOOTH_GS = 0, HZ_SMOOTH_KACZMARZ = 1, HZ_SMOOTH_DIRECT = 2, HZ_SMOOTH_JACOBI = 3,
               HZ_SMOOTH_SOR = 4 } hz_smoother;

/* Kernel forms of a Kaczmarz level (Sec. 4): one launch per colour; the whole level (sweeps,
   residual and full weighting, or correction and sweeps) in one block's shared memory; one launch
   per sweep over halo tiles; the whole level in the shared memory of a thread-block cluster of up
   to 16 blocks (row bands, neighbour rows through distributed shared memory); the whole level in
   global memory by one persistent cooperative launch per pass, with bounded grid-wide barriers
   between the colour phases (single right-hand side only; a barrier wait that runs out ends the
   launch and the solve returns HZ_ETIMEOUT). All five take the same row actions in the same colour
   order with the same fixed-rounding arithmetic, so they give the same bits; they differ in
   launches and parallelism only. */
typedef enum { HZ_KACZ_COLOUR = 0, HZ_KACZ_LEVEL = 1, HZ_KACZ_TILE = 2, HZ_KACZ_CLUSTER = 3, HZ_KACZ_GRID = 4 } hz_kacz_form;

typedef struct {
  int levels;    /* number of grids; 0 = coarsen while n_l is even and larger than 8 */
  int variant;   /* hz_variant, default HZ_VAR_HYB */
  int precision; /* hz_prec, default HZ_PREC_FP64 */
  int nu_gs;     /* Gauss-Seidel pre and post sweeps, default 1 (Sec. 5) */
  int nu_kacz;   /* Kaczmarz pre and post sweeps on the kH ~ 1.25 scale, default 4 (Sec. 5) */
  int guard;     /* 1 (default): an HYB level set to relax with L by the scale bins relaxes with M
                    when some node has 1 < k H < 2 sqrt(2), where red-black GS on L amplifies
                    oscillatory error */
  double k_ref;  /* wavenumber that sets each level's scale c = k_ref H; 0 = mean of k(x) */
  int batch;     /* right-hand sides solved together by hz_solve_batch (1..1024, default 1); every
                    kernel launch then covers all of them and finished ones retire individually */
  int pass_variant; /* kernel form of the two fused passes of each Gauss-Seidel level, in either
                       precision: -1 (default) = chosen per level at setup by timing every form on
                       the level's arrays (tile autotuner; FP64 levels below n_l = 2048 keep
                       tiles); 0 = shared-memory tiles; 1..8 = register streaming with 2^v rows
                       per warp. Every form gives the same bits. */
  int coarse_tail;  /* 1 (default): the smallest levels, from the first whose whole V-cycle below it
                       fits one block's shared memory down to the coarsest, run as one launch (same
                       operations, same results as the per-level kernels for one-sweep Gauss-Seidel
                       and FP32 Kaczmarz levels); 0: one or more launches per level */
  int kacz_form;    /* how Kaczmarz levels below the finest run (hz_kacz_form): -1 (default) = one
                       block if the level fits its shared memory, else tiles with two sweeps per
                       launch (n_l >= 256, sweep count a multiple of 4), else a thread-block
                       cluster, else tiles (even sweep counts), else colour launches in the FP32 form; a cluster,
                       else colour launches in the FP64 form. A form that does not apply to a level
                       falls back to that default. */
  int gs_smoother;  /* smoother of the levels the rules of Sec. 5 give Gauss-Seidel: HZ_SMOOTH_GS
                       (default, red-black), HZ_SMOOTH_JACOBI (damped) or HZ_SMOOTH_SOR (red-black,
                       over-relaxed) -- the alternatives the remark of Sec. 4 names. Jacobi and SOR
                       levels run unfused, one launch per sweep or colour, outside the coarse tail. */
  double omega;     /* relaxation factor of Jacobi or SOR in [0, 2); 0 (default) = 0.8 for Jacobi,
                       1 for SOR (then SOR is Gauss-Seidel) */
  int kacz_rule;    /* which levels relax by Kaczmarz, the normal-equation relaxation Sec. 4 brings in
                       where Gauss-Seidel is no smoother (hz_kacz_rule): HZ_KACZ_RULE_BAND (default)
                       = every level with some node whose k(x) H lies in [0.625 sqrt 2, 2 sqrt 2)
                       (in a heterogeneous medium one level spans k_min H .. k_max H, so several
                       levels can qualify); HZ_KACZ_RULE_BINS = only the levels whose scale
                       c = k_ref H is in the kH ~ 1.25 bin [0.625 sqrt 2, 1.25 sqrt 2). Kaczmarz
                       levels relax with M (HYB, SL) or L (HLM). */
} hz_hierarchy_opts;

typedef enum { HZ_KACZ_RULE_BAND = 0, HZ_KACZ_RULE_BINS = 1 } hz_kacz_rule;

typedef struct {
  int n;        /* n_l */
  double H;     /* 1 / n_l */
  int relax_op; /* hz_op used for relaxation, role (A) of Sec. 5 (the direct-solve operator on the coarsest) */
  int smoother; /* hz_smoother */
  int resid_op; /* hz_op used for the residual, role (B) of Sec. 5 */
  int nu;       /* sweeps before and after the coarse-grid correction */
  int pass_down; /* form of the fused pre-smoothing pass (see pass_variant); -1 = not a fused level
                    or not yet set up */
  int pass_up;   /* form of the fused post-smoothing pass; -1 likewise */
  int in_tail;   /* 1 if the level runs inside the one-block coarse tail (see coarse_tail) */
  int kacz_form; /* hz_kacz_form of a Kaczmarz level outside the tail; -1 otherwise or before setup */
} hz_level_info;

typedef struct {
  double iterations;  /* Bi-CGSTAB iterations; a stop after the half step counts .5 (Table 1) */
  double relres_true; /* |b - A x| / |b| recomputed in FP64 at the stop */
  int history_len;    /* entries written to history: one per half step */
  int status;         /* hz_status of the solve */
  int restarts;       /* restarts after a recurrence residual that the true residual did not confirm */
} hz_solve_info;

/* Fill opts with the defaults listed in hz_hierarchy_opts. */
void hz_default_opts(hz_hierarchy_opts* opts);

/* Create a problem for Eq. 1 on the (n+1)^2 grid.
 *  n       : grid intervals per side, 2 <= n <= 32768.
 *  k_field : host array of (n+1)^2 doubles, wavenumber k(x) > 0 at each node (copied).
 *  beta    : shift of M = L + i k^2 beta (Eq. 3); the paper uses 0.5.
 *  bc      : HZ_BC_SOMMERFELD1.
 *  out     : receives the new problem.
 * Returns HZ_EINVAL on a bad size, non-positive or non-finite k, or a null pointer.
 * Does not touch the device. */
hz_status hz_create_problem(int n, const double* k_field, double beta, int bc, hz_problem** out);

/* Stream for all later work on the problem (a cudaStream_t; NULL = legacy default stream). */
hz_status hz_set_stream(hz_problem* p, void* cuda_stream);

/* Device bytes hz_setup_hierarchy needs for a grid of n intervals and these options (NULL =
 * defaults): level arrays, Krylov vectors, the coarsest inverse and the reduction scratch. */
size_t hz_footprint_bytes(int n, const hz_hierarchy_opts* opts);

/* Build the level hierarchy of Sec. 5 on the device: k injected to each coarse grid,
 * per-level relaxation/residual operators and smoothers, the dense inverse of the coarsest
 * operator. arena: device buffer of at least hz_footprint_bytes bytes, aligned to 256 bytes,
 * owned by the caller and kept alive until hz_destroy; NULL = the library allocates it with
 * cudaMalloc and frees it in hz_destroy. Synchronises the stream. Calling it again rebuilds. */
hz_status hz_setup_hierarchy(hz_problem* p, const hz_hierarchy_opts* opts, void* arena, size_t arena_bytes);

/* The level schedule hz_setup_hierarchy builds for this problem and these options (NULL =
 * defaults): grids, and per level the operators of roles (A) and (B) and the smoother chosen by
 * the variant's rules (Sec. 5). Computed on the host; touches no device. Writes up to cap
 * entries to out (host) and returns the number of levels, or -1 on bad arguments. */
int hz_describe_hierarchy(const hz_problem* p, const hz_hierarchy_opts* opts, hz_level_info* out, int cap);

/* Number of levels (0 before setup) and the description of one level. */
int hz_num_levels(const hz_problem* p);
hz_status hz_get_level_info(const hz_problem* p, int level, hz_level_info* info);

/* z = K r: one V-cycle (Sec. 5) from a zero guess on the finest grid. r, z: device,
 * (n+1)^2 complex128, physical units (z approximates (L^h)^{-1} r). r and z may not alias. */
hz_status hz_vcycle(hz_problem* p, const double* r, double* z);

/* Solve L^h x = rhs by right-preconditioned Bi-CGSTAB (Sec. 6) from x0 = 0 to
 * |rhs - L^h x| / |rhs| <= tol, at most maxit iterations.
 *  rhs, x  : device, (n+1)^2 complex128. x receives the solution (or the last iterate).
 *  history : host, capacity history_cap doubles (may be NULL/0): relative recurrence residual
 *            after every half step.
 *  info    : host, may be NULL.
 * Returns HZ_OK, HZ_EMAXIT (also when the recurrence converged but the true residual never
 * confirmed it, see hz_solve_info.restarts), HZ_EBREAKDOWN or HZ_ENONFINITE (x holds the last
 * iterate), HZ_ETIMEOUT (a bounded wait of the grid-synchronised Kaczmarz form ran out; x is not
 * meaningful), or an argument/CUDA error. Synchronises the stream. */
hz_status hz_solve(hz_problem* p, const double* rhs, double* x, double tol, int maxit,
                   double* history, int history_cap, hz_solve_info* info);

/* Solve for all `batch` right-hand sides of the hierarchy at once (hz_hierarchy_opts.batch):
 * rhs, x: device, batch consecutive (n+1)^2 complex128 vectors. Each right-hand side runs its own
 * Bi-CGSTAB (own scalars, own stop) inside the same kernel launches; one that stops early skips
 * the remaining work. infos: host array of batch entries (may be NULL). Returns HZ_OK when every
 * instance converged, else the first failing instance's status (per-instance status in infos).
 * hz_solve and the non-blocking calls require batch = 1. Synchronises. */
hz_status hz_solve_batch(hz_problem* p, const double* rhs, double* x, double tol, int maxit, hz_solve_info* infos);

/* Groups: several (batched) problems of different grids solved together. Every iteration of
 * every problem is captured into ONE CUDA graph (each problem's kernels on its own branch), and
 * that graph is replayed until every right-hand side of every problem has stopped; finished ones
 * skip their work inside the kernels. The problems must be set up and must not be used elsewhere
 * while the group solves. */
typedef struct hz_group hz_group;
hz_status hz_group_create(hz_problem* const* probs, int count, hz_group** out);
/* rhs[i], x[i]: device, problem i's batch consecutive (n_i+1)^2 complex128 vectors. infos: host,
 * one entry per right-hand side, problem by problem (may be NULL). Synchronises. */
hz_status hz_group_solve(hz_group* g, const double* const* rhs, double* const* x, double tol, int maxit,
                         hz_solve_info* infos);
const char* hz_group_last_error(const hz_group* g);
void hz_group_destroy(hz_group* g);

/* As hz_solve with rhs and x in host memory: copies rhs to the device and x back. */
hz_status hz_solve_host(hz_problem* p, const double* rhs_host, double* x_host, double tol, int maxit,
                        double* history, int history_cap, hz_solve_info* info);

/* ---- Non-blocking solve: one host thread can keep many problems' solves in flight (serving).
 * hz_solve_start validates, copies rhs into the problem's own buffer, queues the start-up and the
 * first iterations (one graph launch each) on the problem's stream and returns; hz_solve_poll
 * never waits: it reads the progress flags that have already landed, queues further iterations
 * (or the true residual, and a restart from it when the recurrence converged without it), and
 * sets *done = 1 once the solve has stopped (converged, broken down, non-finite or maxit). The
 * iterations are launched from the host rather than looped on the device (as hz_solve does)
 * because solves on different streams then overlap on the GPU;
 * hz_solve_finish waits for the end if needed, copies the solution to x and reports exactly as
 * hz_solve does (status, history, info). x holds the result only after hz_solve_finish returns.
 * One solve per problem at a time (HZ_EINVAL otherwise); x must stay valid until
 * hz_solve_finish. A CUDA error during polling ends the solve and is returned. */
hz_status hz_solve_start(hz_problem* p, const double* rhs, double* x, double tol, int maxit);
hz_status hz_solve_poll(hz_problem* p, int* done);
hz_status hz_solve_finish(hz_problem* p, double* history, int history_cap, hz_solve_info* info);

/* ---- Individual steps (the kernels the V-cycle and Bi-CGSTAB run), for testing and for
 * callers that compose their own cycles. All arrays are device complex128 in physical units
 * on level `level`'s grid; they run in the hierarchy's precision. ---- */

/* v = A u on the finest grid with A = L^h (op = HZ_OP_L, Eq. 2) or M^h (HZ_OP_M, Eq. 3), FP64. */
hz_status hz_apply(hz_problem* p, int op, const double* u, double* v);

/* The level's pre-relaxation from a zero guess (nu sweeps of its smoother with its (A)
 * operator: red first for GS, colours 0..4 for Kaczmarz) giving u, then fc = FW(f - B u)
 * with its (B) operator (Sec. 5). fc lives on level+1. Not valid on the coarsest level. */
hz_status hz_level_presmooth(hz_problem* p, int level, const double* f, double* u, double* fc);

/* u = post-relaxation of (u_pre + P ec): bilinear correction from level+1, then nu sweeps
 * (black first for GS, colours 4..0 for Kaczmarz). Not valid on the coarsest level. */
hz_status hz_level_postsmooth(hz_problem* p, int level, const double* f, const double* u_pre,
                              const double* ec, double* u);

/* `sweeps` sweeps of the level's smoother on A u = f starting from the u passed in (in place);
 * post = 0 uses the pre-relaxation ordering, 1 the post ordering. */
hz_status hz_level_sweeps(hz_problem* p, int level, const double* f, double* u, int sweeps, int post);

/* u = A_c^{-1} f on the coarsest level (dense inverse of its operator). */
hz_status hz_coarse_solve(hz_problem* p, const double* f, double* u);

/* ---- Measurement ---- */

/* Kernels of the hot path, as reported by hz_profile_iteration. */
typedef enum {
  HZ_K_GS_FIRST = 0,   /* first red-black half sweep from a zero guess */
  HZ_K_GS_COLOUR,      /* one colour of a red-black Gauss-Seidel sweep */
  HZ_K_KACZ_COLOUR,    /* one colour of a Kaczmarz sweep */
  HZ_K_ZERO,           /* zero fill of a Kaczmarz level's guess */
  HZ_K_RESTRICT,       /* residual with full weighting */
  HZ_K_PROLONG,        /* bilinear correction */
  HZ_K_COARSE,         /* dense solve on the coarsest grid */
  HZ_K_EXPORT,         /* FP32 V-cycle result to the FP64 Krylov vector */
  HZ_K_UPDATE_P,       /* p = r + beta (p - omega v) */
  HZ_K_APPLY_RV,       /* v = A y with <r^, v> */
  HZ_K_UPDATE_S,       /* s = r - alpha v with |s|^2 */
  HZ_K_APPLY_TS,       /* t = A z with <t, s>, <t, t> */
  HZ_K_UPDATE_R,       /* r = s - omega t with <r^, r>, |r|^2 */
  HZ_K_SMOOTH_RESTRICT, /* fused: GS sweep from a zero guess, residual, full weighting */
  HZ_K_PROLONG_SMOOTH, /* fused: bilinear correction and GS post-sweep */
  HZ_K_KACZ_LEVEL,     /* whole Kaczmarz level in one block (pre: sweeps + residual + FW; post: correction + sweeps) */
  HZ_K_KACZ_SWEEP,     /* one five-colour Kaczmarz sweep over halo tiles */
  HZ_K_TAIL,           /* coarse tail: every level from hz_level_info.in_tail down, in one block */
  HZ_K_KACZ_CLUSTER,   /* whole Kaczmarz level over a thread-block cluster (pre or post, as HZ_K_KACZ_LEVEL) */
  HZ_K_JACOBI,         /* one damped Jacobi sweep, out of place */
  HZ_K_KACZ_GRID,      /* whole Kaczmarz level by one cooperative launch (pre or post, as HZ_K_KACZ_LEVEL) */
  HZ_K_UPDATE_X,       /* half of the deferred solution update: x += alpha y or x += omega z */
  HZ_K_COUNT
} hz_kernel;

typedef struct {
  int kernel;  /* hz_kernel */
  int level;   /* grid level the launch works on (0 for the Krylov kernels) */
  float ms;    /* device time between the events recorded around the launch */
} hz_kernel_time;

/* Device time of every kernel launch in `iterations` Bi-CGSTAB iterations of the solve of
 * L^h x = rhs (rhs, x: device), measured with CUDA events recorded on the library's stream
 * around each launch. The iterations are launched one kernel at a time instead of from the
 * CUDA graph; the arithmetic is the same as hz_solve's first iterations. Writes up to cap
 * records to out (host) and returns the number of launches, or -1 on error. Synchronises. */
int hz_profile_iteration(hz_problem* p, const double* rhs, double* x, int iterations, hz_kernel_time* out, int cap);

/* The same records for `iterations` iterations captured as one CUDA graph with an event node
 * after every kernel and replayed once: each record is the time from the previous event node to
 * the kernel's own, i.e. the kernel as it runs inside the solve's graph replay (back to back,
 * with the graph's launch gaps). Synchronises. */
int hz_profile_graph(hz_problem* p, const double* rhs, double* x, int iterations, hz_kernel_time* out, int cap);

/* Diagnostics: the Bi-CGSTAB scalars of one instance after the last solve, as 17 doubles:
 * rho, alpha, omega, beta (complex, re/im pairs), |r|^2, |s|^2, |t|^2, |b|^2 (h^2-scaled), the
 * iteration, the stop code (0 running, 1 converged, 2 breakdown, 3 non-finite, 4 maxit), the
 * smallest |<r^, r>|^2 / (|r^|^2 |r|^2) seen, the number of near-breakdown restarts, and the
 * smallest |omega|^2 |t|^2 / |r|^2 seen in iterations whose |<r^, r>|^2 / (|r^|^2 |r|^2) is below
 * the near-breakdown threshold (see hz_set_stall_detection).
 * Returns 17, or -1 on error. Synchronises. */
int hz_krylov_scalars(hz_problem* p, int instance, double* out);

/* Near-breakdown detection of Bi-CGSTAB (a safeguard the paper does not discuss): after an
 * iteration with |<r^, r>|^2 < cos2 |r^|^2 |r|^2 and |omega|^2 |t|^2 < step2 |r|^2 (the
 * recurrences no longer move r), the shadow residual r^ is renewed with fresh pseudo-random
 * values and the next direction restarts from r, at most max_restarts times per solve. Defaults
 * 1e-12, 1e-8, 16; max_restarts = 0 turns it off. Applies to the solves started after the call.
 * Returns HZ_EINVAL for a negative or non-finite threshold or max_restarts outside [0, 1024]. */
hz_status hz_set_stall_detection(hz_problem* p, double cos2, double step2, int max_restarts);

/* Name of an hz_kernel. */
const char* hz_kernel_name(int kernel);

/* Measured FP64 FMA throughput of the current device (the paper has no counterpart; it sets the
 * roofline of the FP64 Krylov kernels, which GB300's FP64 pipe bounds before HBM): full warps of
 * independent DFMA chains on every SM, `iters` FMAs per chain, timed with CUDA events on `stream`
 * (a cudaStream_t, NULL = legacy default stream), each launch shape (4 or 8 blocks of 256 threads
 * per SM, 8 or 16 chains a thread) after an untimed warm-up launch; the best shape counts. Writes the rate
 * in TFLOP/s (an FMA counts 2 flops) to *tflops (host) and the launch time to *ms (host, may be
 * NULL). Synchronises the stream. Returns HZ_EINVAL for iters outside [1, 2^24] or a null tflops,
 * HZ_ECUDA if a launch or event fails. */
hz_status hz_measure_fp64_rate(int iters, void* stream, double* tflops, double* ms);

/* ---- Allocation-free variant (the paper has no counterpart to this entry point) ----
 * For callers that cannot allocate device memory when they call: hosts whose own pool owns every
 * byte of the device (a framework's caching allocator, a serving runtime's memory budget), where
 * a stray cudaMalloc fragments or oversubscribes the pool, and latency-critical loops, where
 * cudaMalloc and cudaFree may synchronise the device.
 *
 * v = A u on the (n+1)^2 grid (A = L^h for beta = 0, M^h = L^h + i k^2 beta otherwise; physical
 * units, as hz_apply) and dot = <w, v> = sum_p conj(w_p) v_p, in one pass; no problem object.
 *  kh      : device, (n+1)^2 doubles, k(x) h at each node.
 *  u, w, v : device, (n+1)^2 complex128; u and w may be the same array; v shares no byte with
 *            u, w or kh.
 *  dot     : device, one complex128, sharing no byte with v, u, w or kh.
 *  stream  : a cudaStream_t (NULL = legacy default stream); the call is asynchronous on it.
 * Allocates nothing: its only scratch (per-block partial sums and a counter, about 33 KB) is a
 * fixed array in the library's device memory, present on every device that loads the library
 * until the process exits. The first call on a device looks up and caches that array's device
 * address (cudaGetSymbolAddress): make it before any stream capture. Every call shares the array
 * and clears its counter, so calls that overlap on the GPU (other streams or host threads) race
 * and give wrong results: order them. Returns HZ_EINVAL for n outside [2, HZ_NOALLOC_MAX_N], a
 * null pointer or overlapping output and input ranges (nothing launched), HZ_ECUDA if a launch fails. */
#define HZ_NOALLOC_MAX_N 32768
hz_status hz_apply_dot_noalloc(int n, const double* kh, double beta, const double* u, const double* w, double* v,
                               double* dot, void* stream);

/* ---- Ray correction and the stand-alone cycle solver (Sec. 6, Table 7) ----
 * The near-kernel error is written as sum_j exp(i k d_j . x) a_j(x) over the eight directions
 * d_j = (cos j pi/4, sin j pi/4) with smooth ray functions a_j, which are approximated on a coarse
 * ray grid (Sec. 6; the paper leaves the construction to [BL97]). Reading implemented here: the
 * a_j are bilinear on the vertex grid of spacing H = m h, and the correction is the Galerkin
 * projection  x += P (P^H A P)^{-1} P^H r,  where column 8 C + j of P is the bilinear hat of ray
 * node C (C = J (n/m + 1) + I, node (I m, J m)) times the plane wave exp(i k_ref d_j . x), A = L^h
 * of the problem and r = rhs - A x. All of it is complex FP64; P^H A P is assembled and factored on
 * the device (block tridiagonal by rows of ray nodes, block LU with pivoted Gauss-Jordan inverses
 * of the pivot blocks, one refinement step per solve). */
typedef struct hz_ray hz_ray; /* opaque; created by hz_ray_create, freed by hz_ray_destroy */

typedef struct {
  int m;           /* ray grid factor: H = m h */
  int nc;          /* ray cells per side, n / m */
  int unknowns;    /* 8 (nc + 1)^2 */
  double kH;       /* k_ref H */
  size_t bytes;    /* device memory the ray correction holds */
  double setup_ms; /* wall time of hz_ray_create's assembly and factorisation */
} hz_ray_info;

#define HZ_RAY_MAX_NC 128

/* The ray grid factor hz_ray_create takes for m = 0: the largest power of two m with
 * k_ref m / n <= 2.5 that divides n and leaves n / m >= 2 (1 if none larger does). Host only;
 * 0 for n < 2 or a non-positive or non-finite k_ref. */
int hz_ray_spacing(int n, double k_ref);

/* Device bytes of the ray correction of an n-interval grid (m = 0: the factor hz_ray_spacing
 * gives for k_ref): six sets of (nc + 1) blocks of (8 (nc + 1))^2 complex128, the plane-wave table
 * (8 (n+1)^2 complex128) and a few ray vectors; 0 for an invalid n or m. */
size_t hz_ray_footprint_bytes(int n, double k_ref, int m);

/* Build the ray correction of problem p (after hz_setup_hierarchy; uses p's stream and k field).
 *  k_ref : wavenumber of the plane waves, > 0.
 *  m     : ray grid factor, a power of two dividing n with 1 <= n / m <= HZ_RAY_MAX_NC; 0 = the
 *          largest power of two with k_ref m h <= 2.5 (the paper's coarsest scale) that divides n
 *          and leaves at least two ray cells (hz_ray_spacing).
 *  arena : device buffer of at least hz_ray_footprint_bytes bytes, 256-byte aligned, owned by the
 *          caller and kept alive until hz_ray_destroy; NULL = the library allocates it with
 *          cudaMalloc and frees it in hz_ray_destroy.
 *  out   : receives the object; destroy it before p (hz_ray_destroy waits for the device).
 * Synchronises the stream. Returns HZ_EINVAL (bad k_ref, m or arena alignment), HZ_ENOTSETUP,
 * HZ_ENOMEM (arena too small or allocation refused), HZ_EBREAKDOWN (a pivot block of the ray
 * operator is singular) or HZ_ECUDA. */
hz_status hz_ray_create(hz_problem* p, double k_ref, int m, void* arena, size_t arena_bytes, hz_ray** out);
hz_status hz_ray_get_info(const hz_ray* r, hz_ray_info* info);

/* g = P^H res (res: device (n+1)^2 complex128; g: device 8 (nc+1)^2 complex128, ordered 8 C + j).
 * Here and in the calls below an output that shares a byte with an input is refused (HZ_EINVAL). */
hz_status hz_ray_restrict(hz_ray* r, const double* res, double* g);
/* z = (P^H A P)^{-1} g (device, 8 (nc+1)^2 complex128 each, not aliased). */
hz_status hz_ray_coarse_solve(hz_ray* r, const double* g, double* z);
/* Copies of the assembled blocks of P^H A P (before factorisation): device buffers of
 * (nc+1) * (8 (nc+1))^2 complex128 each, block J row-major; lower[J] couples ray row J with row
 * J - 1 (lower[0] is zero), upper[J] with row J + 1 (upper[nc] is zero). Any pointer may be NULL. */
hz_status hz_ray_blocks(hz_ray* r, double* lower, double* diag, double* upper);
/* x += P (P^H A P)^{-1} P^H res (device (n+1)^2 complex128 each, not aliased). */
hz_status hz_ray_correct(hz_ray* r, const double* res, double* x);
void hz_ray_destroy(hz_ray* r);

/* Bytes of scratch hz_cycle_solve needs for an n-interval grid (three (n+1)^2 complex128 vectors
 * and the reduction partials); 0 for n outside [2, 32768]. */
size_t hz_cycle_scratch_bytes(int n);

/* Table 7's stand-alone solver of L^h x = rhs from x = 0: every cycle adds the V-cycle of the
 * residual (hz_vcycle; the hierarchy's variant and precision) and then, when ray is not NULL, the
 * ray correction of the new residual; after each cycle the FP64 residual |rhs - L^h x| / |rhs| is
 * read back and the solve stops when it is <= tol.
 *  rhs, x  : device (n+1)^2 complex128 sharing no byte; x receives the last iterate.
 *  scratch : device buffer of at least hz_cycle_scratch_bytes(n) bytes, 256-byte aligned, owned
 *            by the caller and sharing no byte with rhs or x; NULL = the library allocates and
 *            frees it within the call.
 *  history : host, capacity history_cap (may be NULL/0): the relative residual after each cycle.
 *  info    : host, may be NULL; iterations = cycles, relres_true = the last relative residual.
 * Returns HZ_OK, HZ_EMAXIT (maxc cycles, or the residual grew above 1e8 |rhs|: diverged),
 * HZ_ENONFINITE, or an argument/allocation/CUDA error. One right-hand side (batch 1).
 * Synchronises the stream every cycle. */
hz_status hz_cycle_solve(hz_problem* p, hz_ray* ray, const double* rhs, double* x, double tol, int maxc,
                         void* scratch, size_t scratch_bytes, double* history, int history_cap,
                         hz_solve_info* info);

/* Last error message on p (never NULL), and a name for a status code. */
const char* hz_last_error(const hz_problem* p);
const char* hz_status_string(int status);

/* Free the problem and everything the library allocated for it. Synchronises its stream. */
void hz_destroy(hz_problem* p);

#ifdef __cplusplus
}
#endif

#endif /* HZ_H */
