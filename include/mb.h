/*
 * mb.h — C ABI of the GB300 rigid multiblob mobility library (libmb.so).
 *
 * The library solves the mobility problem of rigid multiblob bodies above a
 * no-slip wall at z = 0 (Balboa Usabiaga et al., "Hydrodynamics of
 * Suspensions of Passive and Active Rigid Particles: A Rigid Multiblob
 * Approach", Sections 2.1-2.2 and 5) on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every call
 *   Arrays are contiguous, row-major, FP64 unless stated: positions r and
 *   blob vectors are N x 3, body vectors n_b x 3, quaternions n_b x 4 with the
 *   scalar first (s, x, y, z), rotation R = (s^2 - v.v) I + 2 v v^T + 2 s [v]x.
 *   Body p owns blobs blob_start[p] .. blob_start[p+1]-1 (int64 CSR offsets).
 *   Units are arbitrary but consistent; a is the blob radius, eta the
 *   viscosity.  wall != 0 adds the single-wall correction, wall == 0 gives the
 *   unbounded-domain RPY mobility.
 *
 *   Pointers are DEVICE pointers owned by the caller unless a call says
 *   otherwise; the library never frees them.  Calls are stream-ordered on the
 *   given stream (a cudaStream_t passed as void*, NULL = legacy default
 *   stream).  Argument errors are detected on the host and returned before
 *   any work is queued.  A context may be used by one host thread and one
 *   stream at a time; it owns all workspace (packed positions, factors,
 *   Krylov basis), grown on demand up to its HBM budget.
 *
 *   Every call returns an mb_status; mb_last_error() gives a message for the
 *   last failing call on a context.  The library never aborts the process.
 */
#ifndef MB_H
#define MB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MB_OK = 0,
    MB_EINVAL = 1,         /* bad argument (null pointer, N < 0, a <= 0 ...) */
    MB_ENOMEM = 2,         /* workspace would exceed the context's HBM budget,
                              or cudaMalloc failed                           */
    MB_ECUDA = 3,          /* a CUDA runtime call failed                      */
    MB_ENOTCONVERGED = 4,  /* Krylov solver hit maxit; best iterate written   */
    MB_ETIMEOUT = 5,       /* a host wait for the stream ran past the limit
                              set by mb_context_set_wait_limit (no kernel of
                              this library waits on the host or on another
                              kernel; the work already enqueued still runs) */
    MB_ESINGULAR = 6       /* a Cholesky factorisation broke down (a body's
                              mobility block not positive definite, e.g. a
                              blob below z = a)                               */
} mb_status;

typedef enum {
    MB_FP64 = 0,          /* pair kernel in FP64                               */
    MB_FP32_KAHAN = 1,    /* pair kernel in FP32 (hi/lo positions, Kahan-
                             compensated accumulation), result in FP64         */
    MB_MIXED_REFINE = 2,  /* solver only: FP32 pair kernel inside the Krylov
                             iteration, double-float pair kernel for the true
                             residual of every restart (iterative refinement)  */
    MB_DF64 = 3           /* pair kernel in double-float: each value an
                             unevaluated sum of two FP32 numbers (~46 bits),
                             FP64-class accuracy (~1e-11 relative) on the FP32
                             pipes, several times faster than MB_FP64 on GB300 */
} mb_precision;

typedef struct mb_context mb_context;

/* Block-diagonal preconditioner (Section 2.2.2).
 *   MB_PRECOND_WALL         each body's own blob mobility block M^(pp),
 *                           including the wall, factorised for every
 *                           configuration (the default);
 *   MB_PRECOND_FREE_SHARED  the blocks of an unbounded domain, which by the
 *                           rotation and translation invariance of the RPY
 *                           tensor depend only on the body's shape: one
 *                           factorisation per shape (bodies with identical
 *                           reference offsets rho), applied to each body by
 *                           rotating the right-hand side into the reference
 *                           frame and the result back (Section 2.2.2).  The
 *                           wall is then left to the Krylov solver: the
 *                           approximate preconditioner of Section 5.4. */
typedef enum { MB_PRECOND_WALL = 0, MB_PRECOND_FREE_SHARED = 1 } mb_precond;

/* Solver parameters.  tol is the target of ||b - A x||_2 / ||b||_2 for the
 * saddle-point system (Eq. saddle_M), measured with the FP64 pair kernel
 * (or FP32 when prec == MB_FP32_KAHAN).  maxit caps the total number of
 * Krylov iterations, restart the Krylov subspace size between restarts.
 * precond selects the preconditioner (mb_solve_mobility only; the batched
 * and serving engines use MB_PRECOND_WALL and reject the other). */
typedef struct {
    double a;
    double eta;
    int wall;
    double tol;
    int maxit;
    int restart;
    mb_precision prec;
    mb_precond precond;
} mb_params;

typedef struct {
    int iters;            /* Krylov iterations (matvecs inside Arnoldi)       */
    int restarts;         /* completed restart cycles                         */
    int converged;        /* 1 if rel_residual <= tol                         */
    double rel_residual;  /* true relative residual of the returned solution  */
    double setup_ms;      /* blob build + preconditioner setup, wall clock    */
    double solve_ms;      /* Krylov solve, wall clock                         */
} mb_info;

/* Human-readable name of a status code (static storage). */
const char *mb_status_string(mb_status s);

/* Message describing the last failing call on ctx (valid until the next
 * call on ctx; "" if none).  With ctx == NULL: the last failing call on this
 * thread that takes no context (mb_context_create,
 * mb_mobility_matvec_noalloc). */
const char *mb_last_error(const mb_context *ctx);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * workspace the context may allocate (0 = 90% of the device's free memory
 * at creation).  *ctx receives the handle. */
mb_status mb_context_create(mb_context **ctx, int device, size_t hbm_budget_bytes);

/* Free the context and all its workspace.  Waits for the device. */
mb_status mb_context_destroy(mb_context *ctx);

/* Bytes of workspace currently held by the context. */
size_t mb_context_workspace_bytes(const mb_context *ctx);

/*
 * Measurement support.  With profiling on, the library brackets every launch
 * of the pair kernel (the O(N^2) direct sum) with CUDA events recorded on the
 * launching stream.  mb_profile_read synchronises on those events and
 * returns the summed pair-kernel time in milliseconds and the number of
 * pair-kernel launches since the last reset; `kernel_launches` receives the
 * number of kernels of any kind this process has launched through the
 * library (a running count, never reset).  reset != 0 clears the recorded
 * events.  Any output pointer may be NULL.
 */
mb_status mb_profile_enable(mb_context *ctx, int on);
mb_status mb_profile_read(mb_context *ctx, double *pair_kernel_ms, int64_t *pair_launches,
                          int64_t *kernel_launches, int reset);

/*
 * Measured FMA rate of the context's device, the roofline denominator of the
 * arithmetic-bound kernels (the pair kernel of Section 5's direct summation
 * and the FP64 factorisations of Section 2.2.2).  prec = MB_FP32_KAHAN
 * measures the FP32 pipe (paired f32x2 FMAs), MB_FP64 the FP64 pipe.  One
 * warm-up and three timed launches of a kernel of independent FMA chains
 * that fills every SM (no memory traffic in its loop); *flops_per_s receives
 * 2 x FMAs / duration of the fastest launch, at the clocks of the moment.
 * Takes about 0.15 s; synchronises the stream.  MB_EINVAL for another
 * precision or a null output.
 */
mb_status mb_measure_fma_rate(mb_context *ctx, mb_precision prec, double *flops_per_s,
                              void *stream);

/*
 * u = M(r) f — product of the blob-blob mobility with blob forces.
 * Section 2.1.1: M_ij is the RPY tensor of Eq. RPYTensor (with its overlap
 * regularisation for r_ij <= 2a; M_ii = I/(6 pi eta a)) plus, if wall != 0,
 * the translation-translation Rotne-Prager-Blake correction for a no-slip
 * wall at z = 0, W(x, y) = eta^-1 (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y) G_img(x, y)
 * with G_img the image part of Blake's Green's function (Eq. MobilityFaxen).
 * Section 5 evaluates this product by O(N^2) direct summation on a GPU; so
 * does this call.
 *
 *   r, f : N x 3 positions and forces (read only)
 *   u    : N x 3 velocities (written)
 *   prec : MB_FP64, MB_FP32_KAHAN or MB_DF64
 * r, f and u may all be device pointers (the call is asynchronous on
 * `stream`) or all host pointers (staged through the context's workspace
 * with copies on `stream`; the call returns after u is written; pinned host
 * memory makes the copies faster).  Mixing kinds is MB_EINVAL.  With the
 * wall, every z must be > 0 (blobs at z < a are computed as written but the
 * matrix need not be positive definite); this is not checked.  N = 0 is a
 * no-op.
 */
mb_status mb_mobility_matvec(mb_context *ctx, const double *r, const double *f, int64_t n,
                             double a, double eta, int wall, mb_precision prec, double *u,
                             void *stream);

/*
 * Choice of the FP32 pair-kernel variant used by this context:
 *   -1  autotune (default): the first FP32 matvec of each size class (half
 *       octaves of N, with or without the wall) runs every variant once on
 *       the caller's stream, synchronises, and keeps the fastest for later
 *       calls — so make that first call before any stream capture;
 *    0  scalar FP32 kernel, one target per thread;
 *    1  packed FP32 kernel (paired f32x2 arithmetic), two targets per thread;
 *    2  packed FP32 kernel, four targets per thread;
 *    3  symmetric packed FP32 kernel: each unordered pair evaluated once
 *       for both blobs (M_ji = M_ij^T), partial sums added to u with FP64
 *       atomics, so results may differ between calls in the last FP64 bits;
 *    4  packed FP32 kernel in 32-thread CTAs (64 targets, source chunks of
 *       32 or more), which spreads small problems over many SMs; the
 *       autotuner's choice below 4,096 blobs.
 * All variants compute the same product to FP32 rounding.  Other values are
 * MB_EINVAL.  Setting a variant clears the autotuner's cache.  Batched
 * solves and servers created on the context use the pinned variant for
 * their FP32 pair launches too (variant 0 runs as 1 there, 4 as 3).
 */
mb_status mb_context_set_pair_variant(mb_context *ctx, int variant);

/* Bound the host waits of mb_solve_mobility, mb_solve_mobility_permeable,
 * mb_solve_resistance, mb_precond_setup and mb_mobility_matvec with host
 * pointers: a wait for the caller's stream (a synchronisation, or the poll
 * of a residual estimate the device posts) that has not finished after
 * `seconds` returns MB_ETIMEOUT instead of blocking.  None of the library's
 * kernels waits on anything, so a wait runs long only behind other work on
 * the stream or a device that stopped answering.  seconds <= 0 (the
 * default) waits without limit.  After MB_ETIMEOUT the work already
 * enqueued on the stream still runs and writes the context's workspace and
 * the call's outputs: the caller synchronises the stream before the next
 * call on this context.  The batched and serving engines keep their waits
 * unbounded (their host bookkeeping follows each wait).  Returns MB_EINVAL
 * for a non-finite limit. */
mb_status mb_context_set_wait_limit(mb_context *ctx, double seconds);

/* The FP32 pair-kernel variant this context uses for N blobs with or
 * without the wall: the fixed variant if one was set, else the autotuner's
 * cached choice for that size class, else -1 (not tuned yet). */
mb_status mb_context_pair_variant(const mb_context *ctx, int64_t n, int wall, int *variant);

/*
 * Allocation-free variant of mb_mobility_matvec with MB_FP32_KAHAN.
 * The paper has no counterpart: this call exists for callers that cannot
 * allocate device memory — applications whose framework owns the whole
 * device-memory budget (its caching allocator has reserved it, so a
 * cudaMalloc would fail or fragment it) and code on latency-critical paths
 * that cannot take cudaMalloc's implicit device synchronisation.
 *
 * It takes no context and allocates nothing (no cudaMalloc, no cudaFree, no
 * allocating library routine).  Its scratch — packed FP32 hi/lo positions
 * and per-chunk partial sums, about 14 MiB — is one file-scope device array
 * of the library, sized for at most MB_NOALLOC_MAX_BLOBS blobs; every GPU
 * that loads the library holds it until the process exits.  Larger N is
 * rejected with MB_EINVAL before anything is queued.
 *
 * The first call on a device (the device current on the calling thread)
 * looks up the array's device address and the device's SM count; make that
 * first call before any stream capture.  All calls share the one array and
 * it keeps the last call's contents; every element a call reads it has
 * written first, so no clearing is needed, but calls whose work overlaps on
 * the GPU (different streams, or host threads) race on it and must be
 * serialised by the caller.
 *
 * r, f, u: N x 3 device pointers on the device current on the calling
 * thread (host pointers and memory of another GPU are MB_EINVAL); the
 * result is the same product as mb_mobility_matvec (up to FP32 rounding
 * order).
 * Errors are reported through mb_last_error(NULL).
 */
#define MB_NOALLOC_MAX_BLOBS 65536
mb_status mb_mobility_matvec_noalloc(const double *r, const double *f, int64_t n, double a,
                                     double eta, int wall, double *u, void *stream);

/*
 * Blob positions r_i = q_p + R(theta_p) rho_i for every blob i of body p
 * (Section 2.1: tracking point q_p and orientation quaternion theta_p of the
 * reference configuration rho).  Device pointers: q (n_b x 3), theta
 * (n_b x 4, need not be normalised: it is normalised on the fly), blob_start
 * (n_b + 1), rho (N x 3) -> r (N x 3), N = blob_start[n_b].  n_blobs must
 * equal blob_start[n_b] (not checked on the device).
 */
mb_status mb_blob_positions(mb_context *ctx, int64_t n_bodies, int64_t n_blobs,
                            const double *q, const double *theta, const int64_t *blob_start,
                            const double *rho, double *r, void *stream);

/*
 * Kinematic map of Eq. noslip_rigid: v_i = U_p + Omega_p x (r_i - q_p) for
 * each blob i of body p.  UO is n_b x 6 (U then Omega per body); v is N x 3.
 */
mb_status mb_K_apply(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                     const double *q, const int64_t *blob_start, const double *UO, double *v,
                     void *stream);

/*
 * Adjoint kinematic map (force and torque balance rows of Eq. rigidSystem):
 * FT_p = (sum_i lambda_i, sum_i (r_i - q_p) x lambda_i) over the blobs of
 * body p.  lambda is N x 3; FT is n_b x 6 (force then torque).
 */
mb_status mb_KT_apply(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                      const double *q, const int64_t *blob_start, const double *lambda,
                      double *FT, void *stream);

/*
 * Block-diagonal preconditioner setup (Section 2.2.2, Eqs.
 * M_tilde_block_diag and indef_block_P): for every body p, assemble its
 * blob mobility block M^(pp) (with the wall if wall != 0), factor it by FP64
 * Cholesky M^(pp) = L L^T, form the 6 x 6 body Schur complement N~_p =
 * (K_p^T M^(pp)-1 K_p)^-1, and keep in the context either the body's
 * explicit inverse of the indefinite block [[M^(pp), -K_p], [-K_p^T, 0]]
 * (applied as one GEMV), or, when there are at least as many bodies as SMs
 * and blocks of more than 160 rows (up to 2,048), the factored form L,
 * L^-1 K_p and N~_p (applied by triangular solves: the same FP64 work per
 * application, a third of the setup's).  r are the blob positions (device,
 * N x 3).  Synchronises the stream; returns MB_ESINGULAR (with the first
 * failing body in mb_last_error) if a block is not positive definite.
 */
mb_status mb_precond_setup(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                           const double *q, const int64_t *blob_start, double a, double eta,
                           int wall, void *stream);

/*
 * Velocity at arbitrary points x (n_points x 3) of the flow driven by forces
 * f on n_blobs blobs at r (Eq. RPYTensor with the wall correction when
 * wall != 0):  u(x_t) = sum_j M(x_t, r_j) f_j, every point treated as a
 * tracer blob of the same radius a.  Points may coincide with blobs (the
 * overlap branch is regular at zero distance); with the wall they must lie
 * above it (z > 0).  prec: MB_FP32_KAHAN or MB_FP64.  Device pointers only.
 */
mb_status mb_mobility_eval(mb_context *ctx, const double *x, int64_t n_points, const double *r,
                           const double *f, int64_t n_blobs, double a, double eta, int wall,
                           mb_precision prec, double *u, void *stream);

/*
 * Flow rendering of Appendix B: every blob i of radius a is replaced by n_sub
 * blobs of radius a_sub at r_i + sub_offsets[k] (n_sub x 3, typically points
 * on the sphere of radius a), each carrying lambda_i / n_sub, and the
 * velocity v(x) of a tracer blob of radius a_sub is evaluated at the points x
 * as with mb_mobility_eval.  Device pointers only.
 */
mb_status mb_render_flow(mb_context *ctx, const double *x, int64_t n_points, const double *r,
                         const double *lambda, int64_t n_blobs, const double *sub_offsets,
                         int n_sub, double a_sub, double eta, int wall, mb_precision prec,
                         double *v, void *stream);

/*
 * First moments of the blob forces, body by body:
 *   S_p[a][b] = sum_{i in p} lambda_i,a (r_i - q_p)_b     (S: n_b x 9, row-major)
 * Its symmetric traceless part is the stresslet of body p (Section 4.1: the
 * stresslet radius R_s under an applied strain slip), its antisymmetric part
 * the torque.  r, lambda: N x 3; q: n_b x 3; blob_start: n_b + 1 (device).
 */
mb_status mb_lambda_moments(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                            const double *q, const int64_t *blob_start, const double *lambda,
                            double *S, void *stream);

/*
 * Set up the shared unbounded-domain preconditioner (MB_PRECOND_FREE_SHARED)
 * for n_b bodies given by their orientations theta (n_b x 4, unit
 * quaternions, scalar first), blob_start (n_b + 1) and reference offsets rho
 * (N x 3), all device arrays.  Bodies whose offsets are identical (same
 * count, bitwise equal values) share one FP64 factorisation of their
 * free-space block M^(pp) and 6 x 6 Schur complement (Section 2.2.2).  The
 * orientations are copied, so the caller's arrays may change afterwards.
 * Synchronises the stream.  MB_EINVAL for malformed blob_start, MB_ENOMEM
 * beyond the context budget, MB_ESINGULAR if a shape's block is not positive
 * definite (mb_last_error names a body of that shape).
 */
mb_status mb_precond_setup_shared(mb_context *ctx, int64_t n_bodies, int64_t n_blobs,
                                  const double *theta, const int64_t *blob_start,
                                  const double *rho, double a, double eta, void *stream);

/*
 * Apply the preconditioner set up by the last mb_precond_setup or
 * mb_precond_setup_shared on ctx:
 * solve [[M~, -K], [-K^T, 0]] [lambda; UO] = [w; g] (Eq. saddle_M_precon)
 * body by body.  w, lambda: N x 3; g, UO: n_b x 6 (device).
 */
mb_status mb_precond_apply(mb_context *ctx, const double *w, const double *g, double *lambda,
                           double *UO, void *stream);

/*
 * Solve the mobility problem (Eq. saddle_M):
 *   [[M, -K], [-K^T, 0]] [lambda; U] = [slip; -F]
 * for the blob constraint forces lambda and the rigid-body motions (U, Omega)
 * by right-preconditioned flexible GMRES with the block-diagonal
 * preconditioner (Section 2.2), initial guess zero, restarted every
 * params->restart iterations on the true residual.
 *
 *   q, theta, blob_start, rho : bodies (device; see mb_blob_positions)
 *   F, T    : n_b x 3 applied forces and torques (device)
 *   slip    : N x 3 apparent slip (Eq. noslip_explicit) or NULL for none
 *   U, Omega: n_b x 3 outputs; lambda: N x 3 output (device)
 *   info    : host struct, may be NULL
 * Synchronises the stream.  Returns MB_ENOTCONVERGED (with the best
 * iterate written) if maxit is reached, MB_ESINGULAR if a body block is not
 * positive definite.
 */
mb_status mb_solve_mobility(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *q,
                            const double *theta, const int64_t *blob_start, const double *rho,
                            const double *F, const double *T, const double *slip,
                            const mb_params *params, double *U, double *Omega, double *lambda,
                            mb_info *info, void *stream);

/*
 * mb_solve_mobility for permeable bodies (Appendix C): the slip of blob i of
 * body p gains -kappa_p / (eta dV_i) lambda_i, which adds
 * shift_i = kappa_p / (eta dV_i) to the three diagonal entries of M for blob
 * i (in the units of M: velocity per force).  shift: N values (device), one
 * per blob, >= 0; zero recovers impermeable bodies.  The per-body blocks of
 * the preconditioner include the shift (params->precond must be
 * MB_PRECOND_WALL).  Otherwise as mb_solve_mobility.
 */
mb_status mb_solve_mobility_permeable(mb_context *ctx, int64_t n_bodies, int64_t n_blobs,
                                     const double *q, const double *theta,
                                     const int64_t *blob_start, const double *rho,
                                     const double *F, const double *T, const double *slip,
                                     const double *shift, const mb_params *params, double *U,
                                     double *Omega, double *lambda, mb_info *info, void *stream);

/*
 * Solve the resistance problem (Eq. resistance_problem):
 *   M lambda = K [U; Omega] + slip,   (F, T) = K^T lambda,
 * for the blob forces lambda that move the bodies rigidly with prescribed
 * velocities (U, Omega), and the forces and torques they add up to
 * (F = R U + R~ slip of Section 2.1.2).  Right-preconditioned GMRES on M with
 * the block-diagonal preconditioner of the blob blocks M^(pp)^-1 (per body
 * with the wall, or shared per shape without it: params->precond); mixed
 * precision refines like mb_solve_mobility.  The iteration count grows with
 * the linear size of the suspension, unlike the mobility problem's
 * (Section 4.4).
 *
 *   q, theta, blob_start, rho : bodies (device; see mb_blob_positions)
 *   U, Omega : n_b x 3 prescribed velocities (device)
 *   slip     : N x 3 apparent slip or NULL
 *   F, T     : n_b x 3 outputs; lambda: N x 3 output (device)
 * Synchronises the stream; errors as mb_solve_mobility.
 */
mb_status mb_solve_resistance(mb_context *ctx, int64_t n_bodies, int64_t n_blobs,
                              const double *q, const double *theta, const int64_t *blob_start,
                              const double *rho, const double *U, const double *Omega,
                              const double *slip, const mb_params *params, double *F, double *T,
                              double *lambda, mb_info *info, void *stream);

/* One independent problem of a batch (all pointers device pointers; layout
 * as for mb_solve_mobility; slip may be NULL). */
typedef struct {
    int64_t n_bodies;
    int64_t n_blobs;
    const double *q;
    const double *theta;
    const int64_t *blob_start;
    const double *rho;
    const double *F;
    const double *T;
    const double *slip;
    double *U;
    double *Omega;
    double *lambda;
} mb_problem;

/*
 * Solve many independent mobility problems (Eq. saddle_M, one per problem)
 * together, on the serving engine below with every problem admitted at once.  All problems share `params` (a, eta, wall, tolerance,
 * iteration limits, precision).  The blob build, K, K^T and the block-
 * diagonal preconditioner of Section 2.2.2 run over all bodies of all
 * problems in one launch each; the pair kernel runs as one persistent launch
 * over all problems' (target block, source chunk) work items, so problems of
 * very different sizes share the GPU; each problem keeps its own GMRES
 * state and stops consuming pair-kernel work once converged.  The first
 * FP32 matvec times the packed kernel with 2 and 4 targets per thread and
 * the symmetric kernel (each unordered pair once for both blobs) and keeps
 * the fastest (autotuned tile shape).  The arena is sized exactly for
 * the batch.
 *
 * problems: host array of n_problems descriptors (pointing to device data);
 * infos: host array of n_problems (may be NULL), filled per problem
 * (setup_ms and solve_ms are the batch's).  Synchronises the stream.
 * Returns MB_ENOTCONVERGED if any problem missed the tolerance (each
 * problem's best iterate is written and its info says which), MB_ESINGULAR
 * naming the problem and body whose block is not positive definite, and
 * MB_EINVAL for a malformed descriptor (including blob_start[0] != 0 or
 * blob_start[n_b] != N, detected on the device).
 */
mb_status mb_solve_batch(mb_context *ctx, int n_problems, const mb_problem *problems,
                         const mb_params *params, mb_info *infos, void *stream);

/*
 * Serving: a continuous-batching engine for mobility solves.
 *
 * The server owns one device arena, sized at creation by `limits` and
 * charged to the context's HBM budget: blob and body slots, preconditioner
 * storage and the Krylov basis of restart length params->restart.  Requests
 * (mb_problem descriptors, device pointers that must stay valid until the
 * request completes) are queued by mb_server_submit and admitted when their
 * blobs, bodies and preconditioner blocks fit in the arena (admission by HBM
 * footprint) and a request slot is free.  The queue is scanned in arrival
 * order and every request that fits is admitted, so small requests are not
 * held up behind a large one waiting for room; a request that later ones
 * have overtaken limits->max_bypass times stops the scan until it is
 * admitted itself, which bounds its wait (aging).  Each
 * mb_server_step is one scheduling tick: it retires finished requests
 * (writing U, Omega and lambda to the request's arrays and freeing its
 * ranges), admits queued ones (blob build, preconditioner factorisation,
 * right-hand side), computes the true residual of every request starting a
 * restart cycle, and runs one Arnoldi step of the flexible GMRES of
 * mb_solve_mobility for every active request — all requests share the same
 * kernel launches whatever their size or iteration.  Requests submitted
 * while others are in flight join at the next tick.  A request's result does
 * not depend on which others share its ticks (up to the solver tolerance).
 *
 * A request whose FP32 Arnoldi matvec exceeds limits->tick_pairs pair
 * evaluations has it split over consecutive ticks (the symmetric kernel
 * accumulates the parts); its other steps run once, on the first or the last
 * of those ticks.  Results do not depend on the split.
 *
 * mb_server_step synchronises `stream` once per tick and reports how many
 * requests are running and queued.  mb_server_poll gives a request's state
 * (0 queued, 1 running, 2 done, 3 failed), its info (setup_ms = time from
 * submission to admission, solve_ms = admission to completion) and its
 * status (MB_OK, MB_ENOTCONVERGED, MB_ESINGULAR, MB_EINVAL).  A request too
 * large for the arena is refused at submission with MB_ENOMEM.
 */
typedef struct mb_server mb_server;

typedef struct {
    int64_t max_blobs;          /* blob slots in the arena                   */
    int64_t max_bodies;         /* body slots                                */
    int64_t max_precond_bytes;  /* storage for the bodies' preconditioner
                                   blocks: (3 n_p + 6)^2 doubles per body    */
    int max_requests;           /* requests in flight at once                */
    double tick_pairs;          /* pair evaluations one request may take per
                                   tick in the FP32 Arnoldi matvec (symmetric
                                   tile shape): larger requests spread each
                                   matvec over several ticks, so that small
                                   requests sharing the ticks are not held up
                                   by them; 0 = 1e9 (about 2 ms of the FP32
                                   kernel), < 0 = no limit */
    int max_bypass;             /* admissions of later requests a queued
                                   request may be overtaken by before the
                                   scan stops at it: 0 = 64, < 0 = strict
                                   first-come first-served */
} mb_server_limits;

mb_status mb_server_create(mb_context *ctx, const mb_params *params,
                           const mb_server_limits *limits, mb_server **server);
mb_status mb_server_destroy(mb_server *server);
mb_status mb_server_submit(mb_server *server, const mb_problem *problem, int64_t *ticket);
mb_status mb_server_step(mb_server *server, void *stream, int *n_running, int *n_queued);
mb_status mb_server_poll(mb_server *server, int64_t ticket, int *state, mb_info *info,
                         mb_status *result);

/* Tickets of the requests that finished (done or failed) since the last
 * call, oldest first: up to max_tickets of them are written to `tickets`
 * (host array) and *count receives how many; the rest stay for the next
 * call.  Lets a caller with many requests in flight poll only those. */
mb_status mb_server_finished(mb_server *server, int64_t *tickets, int max_tickets, int *count);

#ifdef __cplusplus
}
#endif

#endif /* MB_H */
