// Internal declarations shared by the translation units of libmb.so.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <map>
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mb.h"

namespace mb {

// A grow-only device buffer owned by a context.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Everything a captured Arnoldi step of the single-problem solver bakes in:
// the context's allocation generation (any workspace reallocation changes
// it), the step index and sizes, the scalars of the kernels and the caller
// and workspace pointers they read.
struct IterSig {
    uint64_t gen = 0;
    int j = -1, m = 0, inner = 0, wall = 0, variant = 0, pc_max_np = 0, pc_kind = 0, mode = 0,
        pc_factored = 0;
    const void *shift = nullptr;
    int64_t n = 0, nb = 0, L = 0, pc_nb = 0;
    double a = 0.0, eta = 0.0;
    const void *q = nullptr, *V = nullptr, *Z = nullptr, *sm = nullptr;
    bool operator==(const IterSig &o) const
    {
        return gen == o.gen && j == o.j && m == o.m && inner == o.inner && wall == o.wall &&
               variant == o.variant && pc_max_np == o.pc_max_np && pc_kind == o.pc_kind &&
               mode == o.mode && pc_factored == o.pc_factored && shift == o.shift &&
               n == o.n && nb == o.nb &&
               L == o.L && pc_nb == o.pc_nb && a == o.a && eta == o.eta && q == o.q &&
               V == o.V && Z == o.Z && sm == o.sm;
    }
};

// One Arnoldi step captured as a CUDA graph.  A step is captured the second
// time it is met with the same signature (the first run sizes every buffer
// and settles the autotuner) and replayed from then on.
struct IterGraph {
    IterSig sig;
    bool seen = false;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;  // kernels in the graph (launch accounting)
    uint64_t last_use = 0;   // for least-recently-used eviction
};
constexpr size_t kMaxIterGraphs = 256;  // cached steps per context

}  // namespace mb

struct mb_context {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;   // HBM bytes the context may hold
    size_t held = 0;     // bytes currently allocated
    std::string err;

    // matvec workspace
    mb::DevBuf pos_hi, pos_lo;   // packed float4 positions (FP32 path)
    mb::DevBuf partial;          // per-source-chunk partial velocities (FP64)
    mb::DevBuf stage_r, stage_f, stage_u;  // staging for host-pointer calls
    mb::DevBuf eval_hi, eval_lo;           // packed flow-evaluation points (FP32 path)
    mb::DevBuf render_r, render_f;         // refined blobs of a flow rendering
    // spatial order for the symmetric FP32 kernel (matvec_pack_positions):
    // permutation, its sorted packed positions, the bounding box of every
    // block of the kernel, per-cell counters, the grid and far threshold,
    // and the gathered forces / scattered velocities of a matvec
    mb::DevBuf sort_perm, sort_key, sort_count, sort_hi, sort_lo, sort_box, sort_grid;
    mb::DevBuf sort_f, sort_u;
    int64_t sorted_n = 0;                  // N of the current order (0: none)

    // preconditioner (last mb_precond_setup / mb_precond_setup_shared)
    mb::DevBuf pinv;             // explicit inverses, (3n_p+6)^2 doubles each: one per
                                 // body (wall kind) or one per body shape (shared kind)
    mb::DevBuf pinv32;           // FP32 copy of the explicit blocks (FP32 inner iterations)
    mb::DevBuf pinv_off;         // int64 offsets into pinv (bodies or shapes, + 1)
    mb::DevBuf blob_start_copy;  // int64 copy of blob_start used by apply
    mb::DevBuf flag;             // int status flags written by kernels
    mb::DevBuf pc_type;          // shared kind: int shape index of every body
    mb::DevBuf pc_theta;         // shared kind: copy of the bodies' quaternions
    mb::DevBuf pc_ref;           // shared kind: reference positions, zero centres,
                                 // CSR offsets of the shapes (setup input)
    int64_t pc_nb = 0, pc_n = 0;
    int pc_max_np = 0;
    int pc_kind = 0;             // mb_precond of the current blocks
    int pc_schur = 1;            // 0: blocks hold M_pp^-1 only (resistance problem)
    int pc_factored = 0;         // 1: blocks hold L, G = L^-1 K and -N (applied by
                                 // triangular solves), 0: explicit inverses
    int64_t pc_shapes = 0;       // shared kind: distinct shapes
    int64_t pc_doubles = 0;      // entries of the explicit wall blocks in pinv
    bool pc_f32_ready = false;   // pinv32 holds the current explicit blocks in FP32

    // solver workspace
    mb::DevBuf sol_r;            // blob positions
    mb::DevBuf sol_V, sol_Z;     // Krylov bases (restart+1 and restart vectors)
    mb::DevBuf sol_b, sol_x, sol_w, sol_t; // rhs, iterate, scratch vectors
    mb::DevBuf sol_dx, sol_ym;   // mixed precision: cycle correction, running M lambda
    mb::DevBuf sol_small;        // Hessenberg, Givens, dots (doubles)
    mb::DevBuf sol_dots;         // Cholesky scratch of the preconditioner setup
    mb::DevBuf sol_V32;          // FP32 copy of the Krylov basis (small systems, FP32 passes)
    mb::DevBuf sol_body;         // int body of every blob (small-system steps)
    mb::DevBuf batch_ws;         // batched-solve workspace (mb_solve_batch)
    void *host_small = nullptr;  // pinned host mirror of small scalars
    // Arnoldi-step estimates posted by the small-system orthogonalisation:
    // mapped pinned host memory [est, step count] with its device alias, the
    // step count kept on the device, and the count the host last asked for
    double *host_post = nullptr, *host_post_dev = nullptr;
    unsigned long long *post_seq_dev = nullptr;
    unsigned long long post_seq = 0;

    uint64_t alloc_gen = 0;             // bumped by every workspace (re)allocation
    std::vector<mb::IterGraph> iter_graphs;  // captured Arnoldi steps (any problem, any step)
    uint64_t graph_clock = 0;
    cudaStream_t cap_stream = nullptr;       // private stream for captures (the caller's
                                             // stream may be the legacy one)

    // FP32 pair-kernel variant: -1 = autotune per (size class, wall), else fixed
    double wait_limit_s = 0.0;  // host waits for the stream: <= 0 without limit
    int pair_variant = -1;
    std::map<int, int> tuned;   // size-class key -> fastest variant

    // measurement: events around pair-kernel launches (mb_profile_*)
    int profiling = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_used, ev_free;
};

namespace mb {

mb_status set_err(mb_context *ctx, mb_status s, const char *fmt, ...);
// Message for calls without a context (read back by mb_last_error(NULL)).
void set_thread_err(const char *msg);
mb_status cuda_err(mb_context *ctx, cudaError_t e, const char *what);
// Wait for stream s, within the context's wait limit (MB_ETIMEOUT past it).
mb_status wait_stream(mb_context *ctx, cudaStream_t s, const char *what);
// Make `buf` hold at least `bytes`; respects the context budget.
mb_status ensure(mb_context *ctx, DevBuf &buf, size_t bytes, const char *what);
void release(mb_context *ctx, DevBuf &buf);

// Pair matvec on device pointers (implemented in pair_matvec.cu).
// f_stride_blob lets the solver pass its packed vectors (stride 3 doubles).
mb_status matvec_device(mb_context *ctx, const double *r, const double *f, int64_t n, double a,
                        double eta, int wall, mb_precision prec, double *u, cudaStream_t s);
// Autotuner size class of an FP32 matvec (pair_matvec.cu).
int tune_key(int64_t n, int wall);
// Pack positions once (FP32 path); the matvec then only reads f.  order: also
// sort them spatially for the symmetric FP32 kernel (N >= 16,384).
mb_status matvec_pack_positions(mb_context *ctx, const double *r, int64_t n, cudaStream_t s,
                                bool order = true);
// u(x_t) = sum_j M(x_t, r_j) f_j at nt points x (targets) from ns blobs.
mb_status matvec_eval(mb_context *ctx, const double *x, int64_t nt, const double *r,
                      const double *f, int64_t ns, double a, double eta, int wall,
                      mb_precision prec, double *u, cudaStream_t s);
// Appendix B flow rendering: blobs refined into n_sub blobs of radius a_sub.
mb_status render_flow(mb_context *ctx, const double *x, int64_t nt, const double *r,
                      const double *lam, int64_t n, const double *off, int n_sub, double a_sub,
                      double eta, int wall, mb_precision prec, double *v, cudaStream_t s);
// Chunk partial sums of a matvec whose final reduction the caller takes
// over: u = scale * sum_{s < S} partial[s * 3N + e].  S = 0 means that the
// matvec wrote u itself (one chunk, or a kernel without chunks).
// Body of blob i (blob_start ascending, nb bodies), by bisection.
__device__ __forceinline__ int64_t body_of(const int64_t *__restrict__ start, int64_t nb, int64_t i)
{
    int64_t lo = 0, hi = nb;  // invariant: start[lo] <= i < start[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (start[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

struct MatvecPartials {
    const double *partial = nullptr;
    int S = 0;
    double scale = 0.0;
};
// defer (optional): when the chosen kernel writes chunk partials, leave u
// unwritten and describe the partials there instead of reducing them.
mb_status matvec_packed(mb_context *ctx, const double *r, const double *f, int64_t n, double a,
                        double eta, int wall, mb_precision prec, double *u, cudaStream_t s,
                        MatvecPartials *defer = nullptr);

// Bodies (bodies.cu)
mb_status blob_positions(mb_context *ctx, int64_t nb, int64_t n, const double *q,
                         const double *theta, const int64_t *blob_start, const double *rho,
                         double *r, cudaStream_t s);
// v = alpha * K UO + beta * v   (v: N x 3)
void launch_K_apply(int64_t nb, int64_t n, const double *r, const double *q,
                    const int64_t *blob_start, const double *UO, double *v, double alpha,
                    double beta, cudaStream_t s);
// S_p = sum_i lambda_i (x) (r_i - q_p)   (S: n_b x 9, row-major 3 x 3)
void launch_moments(int64_t nb, const double *r, const double *q, const int64_t *blob_start,
                    const double *lambda, double *S, cudaStream_t s);
// FT = alpha * K^T lambda      (FT: n_b x 6)
void launch_KT_apply(int64_t nb, const double *r, const double *q, const int64_t *blob_start,
                     const double *lambda, double *FT, double alpha, cudaStream_t s);
// The rows of the saddle operator of Eq. saddle_M in one launch, from the
// deferred chunk sums of M lambda: with x = [lambda; U],
//   y[0, 3N)          = scale * sum_s partial[s] - K U
//   y[3N, 3N + 6 n_b) = -K^T lambda
// the arithmetic of reduce_partials_kernel followed by K_apply and the
// one-CTA-per-body K^T.  For 1 <= nb <= kSaddleRowsMaxBodies.
constexpr int64_t kSaddleRowsMaxBodies = 256;
void launch_saddle_rows(const MatvecPartials &mp, int64_t n, int64_t nb, const double *r,
                        const double *q, const int64_t *blob_start, const double *x, double *y,
                        cudaStream_t s);

// Preconditioner (precond.cu)
// schur = 0 keeps only the blob blocks M_pp^-1 (resistance problem).
// shift (N per-blob values or null) is added to the diagonal of each M_pp
// (permeable bodies, Appendix C).
mb_status precond_setup(mb_context *ctx, int64_t nb, int64_t n, const double *r,
                        const double *q, const int64_t *blob_start, double a, double eta,
                        int wall, cudaStream_t s, int schur = 1, const double *shift = nullptr);
// Asynchronous setup of the blocks of nb bodies: start (nb+1, global blob
// indices), poff (nb offsets into P); a failing body sets flags[flag_slot] = 2.
mb_status precond_setup_range(mb_context *ctx, int64_t nb, const double *r, const double *q,
                              const int64_t *start, const int64_t *poff, double *P, int max_np,
                              double a, double eta, int wall, int *flags, int flag_slot,
                              cudaStream_t s, int schur = 1);
// Shared unbounded-domain blocks, one per body shape (precond.cu).
mb_status precond_setup_shared(mb_context *ctx, int64_t nb, int64_t n, const double *theta,
                               const int64_t *blob_start, const double *rho, double a,
                               double eta, cudaStream_t s, int schur = 1);
// z = P^-1 v where v = [w (3N); g (6 n_b)] packed contiguously, same for z.
// f32: from the FP32 copy of the explicit blocks when precond_make_f32 made one
void precond_apply_packed(mb_context *ctx, const double *v, double *z, cudaStream_t s,
                          bool f32 = false);
mb_status precond_make_f32(mb_context *ctx, cudaStream_t s);
// z = M~^-1 w with the blob blocks alone (w, z: 3N), for the resistance problem.
void precond_apply_blobs(mb_context *ctx, const double *w, double *z, cudaStream_t s);

// Solver (gmres.cu)
// Eq. resistance_problem: M lambda = K [U; Omega] + slip, then (F, T) = K^T lambda.
mb_status solve_resistance(mb_context *ctx, int64_t nb, int64_t n, const double *q,
                           const double *theta, const int64_t *blob_start, const double *rho,
                           const double *U, const double *Omega, const double *slip,
                           const mb_params *p, double *F, double *T, double *lambda,
                           mb_info *info, cudaStream_t s);
// shift: N per-blob additions to the diagonal of M (kappa_p / (eta dV_i),
// permeable bodies, Appendix C) or null.
mb_status solve_mobility(mb_context *ctx, int64_t nb, int64_t n, const double *q,
                         const double *theta, const int64_t *blob_start, const double *rho,
                         const double *F, const double *T, const double *slip,
                         const mb_params *p, double *U, double *Omega, double *lambda,
                         mb_info *info, cudaStream_t s, const double *shift = nullptr);

// Batched solves on the serving engine (server.cu)
mb_status solve_batch(mb_context *ctx, int np, const mb_problem *probs, const mb_params *prm,
                      mb_info *infos, cudaStream_t s);

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Pair-kernel precision inside the Krylov iteration and for the restart
// residual of each solver precision mode.
inline mb_precision inner_precision(mb_precision p)
{
    return p == MB_FP64 ? MB_FP64 : (p == MB_DF64 ? MB_DF64 : MB_FP32_KAHAN);
}
inline mb_precision outer_precision(mb_precision p)
{
    return p == MB_FP64 ? MB_FP64 : (p == MB_FP32_KAHAN ? MB_FP32_KAHAN : MB_DF64);
}

// Running count of kernels launched through the library (mb_profile_read).
extern std::atomic<long long> g_launches;
inline void count_launch(long long k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Event pair bracketing one pair-kernel launch when profiling is on.
std::pair<cudaEvent_t, cudaEvent_t> *profile_begin(mb_context *ctx, cudaStream_t s);
void profile_end(std::pair<cudaEvent_t, cudaEvent_t> *ev, cudaStream_t s);

}  // namespace mb

#define MB_CUDA_TRY(ctx, call)                                   \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return mb::cuda_err((ctx), e_, #call); \
    } while (0)

#define MB_TRY(call)                       \
    do {                                   \
        mb_status s_ = (call);             \
        if (s_ != MB_OK) return s_;        \
    } while (0)
