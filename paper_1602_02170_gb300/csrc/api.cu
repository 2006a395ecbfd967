// C ABI of libmb.so (declared in include/mb.h): argument checks, context and
// workspace management, host-pointer staging, dispatch to the kernels.
#include <chrono>
#include <cmath>
#include <new>
#include <thread>

#include <initializer_list>

#include "mb_internal.cuh"

namespace mb {

mb_status set_err(mb_context *ctx, mb_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return s;
}

mb_status cuda_err(mb_context *ctx, cudaError_t e, const char *what)
{
    return set_err(ctx, e == cudaErrorMemoryAllocation ? MB_ENOMEM : MB_ECUDA, "%s: %s (%s)", what,
                   cudaGetErrorName(e), cudaGetErrorString(e));
}

mb_status wait_stream(mb_context *ctx, cudaStream_t s, const char *what)
{
    if (!(ctx->wait_limit_s > 0.0)) {
        const cudaError_t e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? MB_OK : cuda_err(ctx, e, what);
    }
    // poll: spin for the first 100 us (short steps), then sleep between queries
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(s);
        if (e == cudaSuccess) return MB_OK;
        if (e != cudaErrorNotReady) return cuda_err(ctx, e, what);
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > ctx->wait_limit_s)
            return set_err(ctx, MB_ETIMEOUT,
                           "%s: the stream had not finished after %.3g s (wait limit); the "
                           "enqueued work still runs, synchronise the stream before the next call",
                           what, ctx->wait_limit_s);
        if (el > 1e-4) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

mb_status ensure(mb_context *ctx, DevBuf &buf, size_t bytes, const char *what)
{
    if (bytes == 0) bytes = 16;
    if (buf.bytes >= bytes) return MB_OK;
    const size_t grow = bytes + bytes / 8;  // headroom against repeated growth
    if (ctx->held - buf.bytes + grow > ctx->budget)
        return set_err(ctx, MB_ENOMEM, "%s: %zu bytes would exceed the HBM budget (%zu held of %zu)",
                       what, grow, ctx->held - buf.bytes, ctx->budget);
    ++ctx->alloc_gen;  // captured graphs that hold the old pointer are stale
    if (buf.ptr) {
        cudaFree(buf.ptr);
        ctx->held -= buf.bytes;
        buf.ptr = nullptr;
        buf.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&buf.ptr, grow);
    if (e != cudaSuccess) {
        buf.ptr = nullptr;
        return cuda_err(ctx, e, what);
    }
    buf.bytes = grow;
    ctx->held += grow;
    return MB_OK;
}

void release(mb_context *ctx, DevBuf &buf)
{
    ++ctx->alloc_gen;
    if (buf.ptr) {
        cudaFree(buf.ptr);
        ctx->held -= buf.bytes;
    }
    buf.ptr = nullptr;
    buf.bytes = 0;
}

mb_status precond_apply_public(mb_context *ctx, const double *w, const double *g, double *lam,
                               double *UO, cudaStream_t s);

std::atomic<long long> g_launches{0};

std::pair<cudaEvent_t, cudaEvent_t> *profile_begin(mb_context *ctx, cudaStream_t s)
{
    if (!ctx->profiling) return nullptr;
    std::pair<cudaEvent_t, cudaEvent_t> ev{nullptr, nullptr};
    if (!ctx->ev_free.empty()) {
        ev = ctx->ev_free.back();
        ctx->ev_free.pop_back();
    } else if (cudaEventCreate(&ev.first) != cudaSuccess ||
               cudaEventCreate(&ev.second) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    ctx->ev_used.push_back(ev);
    cudaEventRecord(ev.first, s);
    return &ctx->ev_used.back();
}

void profile_end(std::pair<cudaEvent_t, cudaEvent_t> *ev, cudaStream_t s)
{
    if (ev) cudaEventRecord(ev->second, s);
}

namespace {

// Device pointer (true), host pointer (false); error on failure.
mb_status pointer_kind(mb_context *ctx, const void *p, bool *device)
{
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_err(ctx, e, "cudaPointerGetAttributes");
    }
    *device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
    return MB_OK;
}

mb_status check_ctx(mb_context *ctx)
{
    if (!ctx) return MB_EINVAL;
    ctx->err.clear();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
    return MB_OK;
}

bool bad_phys(double a, double eta) { return !(a > 0.0) || !(eta > 0.0) || !std::isfinite(a) || !std::isfinite(eta); }

}  // namespace
}  // namespace mb

using namespace mb;

static thread_local std::string g_create_err;

namespace mb {
void set_thread_err(const char *msg) { g_create_err = msg; }
}  // namespace mb

extern "C" {

const char *mb_status_string(mb_status s)
{
    switch (s) {
    case MB_OK: return "MB_OK";
    case MB_EINVAL: return "MB_EINVAL";
    case MB_ENOMEM: return "MB_ENOMEM";
    case MB_ECUDA: return "MB_ECUDA";
    case MB_ENOTCONVERGED: return "MB_ENOTCONVERGED";
    case MB_ETIMEOUT: return "MB_ETIMEOUT";
    case MB_ESINGULAR: return "MB_ESINGULAR";
    }
    return "MB_UNKNOWN";
}


const char *mb_last_error(const mb_context *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

mb_status mb_context_create(mb_context **out, int device, size_t hbm_budget_bytes)
{
    g_create_err.clear();
    if (!out) return MB_EINVAL;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        g_create_err = "no such CUDA device";
        return e != cudaSuccess ? MB_ECUDA : MB_EINVAL;
    }
    if ((e = cudaSetDevice(device)) != cudaSuccess) {
        g_create_err = cudaGetErrorString(e);
        return MB_ECUDA;
    }
    mb_context *ctx = new (std::nothrow) mb_context();
    if (!ctx) return MB_ENOMEM;
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        hbm_budget_bytes = (size_t)(0.9 * (double)fr);
    }
    ctx->budget = hbm_budget_bytes;
    *out = ctx;
    return MB_OK;
}

mb_status mb_context_destroy(mb_context *ctx)
{
    if (!ctx) return MB_EINVAL;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    DevBuf *bufs[] = {&ctx->pos_hi, &ctx->pos_lo, &ctx->partial, &ctx->stage_r, &ctx->stage_f,
                      &ctx->stage_u, &ctx->pinv, &ctx->pinv32, &ctx->pinv_off, &ctx->blob_start_copy,
                      &ctx->flag, &ctx->sol_r, &ctx->sol_V, &ctx->sol_Z, &ctx->sol_b,
                      &ctx->sol_x, &ctx->sol_w, &ctx->sol_t, &ctx->sol_small, &ctx->sol_dots,
                      &ctx->sol_body, &ctx->sol_V32,
                      &ctx->sol_dx, &ctx->sol_ym, &ctx->pc_type, &ctx->pc_theta, &ctx->pc_ref,
                      &ctx->eval_hi, &ctx->eval_lo, &ctx->render_r, &ctx->render_f,
                      &ctx->sort_perm, &ctx->sort_key, &ctx->sort_count, &ctx->sort_hi,
                      &ctx->sort_lo, &ctx->sort_box, &ctx->sort_grid, &ctx->sort_f, &ctx->sort_u,
                      &ctx->batch_ws};
    for (auto &g : ctx->iter_graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (DevBuf *b : bufs) release(ctx, *b);
    if (ctx->host_small) cudaFreeHost(ctx->host_small);
    if (ctx->host_post) cudaFreeHost(ctx->host_post);
    if (ctx->post_seq_dev) cudaFree(ctx->post_seq_dev);
    for (auto &e : ctx->ev_used) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    for (auto &e : ctx->ev_free) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    delete ctx;
    return MB_OK;
}

size_t mb_context_workspace_bytes(const mb_context *ctx) { return ctx ? ctx->held : 0; }

mb_status mb_context_set_wait_limit(mb_context *ctx, double seconds)
{
    MB_TRY(check_ctx(ctx));
    if (!std::isfinite(seconds)) return set_err(ctx, MB_EINVAL, "wait limit must be finite");
    ctx->wait_limit_s = seconds;
    return MB_OK;
}

mb_status mb_context_set_pair_variant(mb_context *ctx, int variant)
{
    MB_TRY(check_ctx(ctx));
    if (variant < -1 || variant > 4) return set_err(ctx, MB_EINVAL, "pair variant must be -1..4");
    ctx->pair_variant = variant;
    ctx->tuned.clear();
    return MB_OK;
}

mb_status mb_context_pair_variant(const mb_context *ctx, int64_t n, int wall, int *variant)
{
    if (!ctx || !variant) return MB_EINVAL;
    if (ctx->pair_variant >= 0) {
        *variant = ctx->pair_variant;
        return MB_OK;
    }
    auto it = ctx->tuned.find(tune_key(n, wall));
    *variant = it == ctx->tuned.end() ? -1 : it->second;
    return MB_OK;
}

mb_status mb_profile_enable(mb_context *ctx, int on)
{
    MB_TRY(check_ctx(ctx));
    ctx->profiling = on ? 1 : 0;
    return MB_OK;
}

mb_status mb_profile_read(mb_context *ctx, double *pair_kernel_ms, int64_t *pair_launches,
                          int64_t *kernel_launches, int reset)
{
    MB_TRY(check_ctx(ctx));
    double total = 0.0;
    for (auto &e : ctx->ev_used) {
        MB_CUDA_TRY(ctx, cudaEventSynchronize(e.second));
        float ms = 0.f;
        MB_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e.first, e.second));
        total += ms;
    }
    if (pair_kernel_ms) *pair_kernel_ms = total;
    if (pair_launches) *pair_launches = (int64_t)ctx->ev_used.size();
    if (kernel_launches) *kernel_launches = (int64_t)g_launches.load();
    if (reset) {
        for (auto &e : ctx->ev_used) ctx->ev_free.push_back(e);
        ctx->ev_used.clear();
    }
    return MB_OK;
}

mb_status mb_mobility_matvec(mb_context *ctx, const double *r, const double *f, int64_t n,
                             double a, double eta, int wall, mb_precision prec, double *u,
                             void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n < 0) return set_err(ctx, MB_EINVAL, "N must be >= 0");
    if (bad_phys(a, eta)) return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (prec != MB_FP64 && prec != MB_FP32_KAHAN && prec != MB_DF64)
        return set_err(ctx, MB_EINVAL, "matvec precision must be MB_FP64, MB_FP32_KAHAN or MB_DF64");
    if (n == 0) return MB_OK;
    if (!r || !f || !u) return set_err(ctx, MB_EINVAL, "null array pointer");
    if (n > (int64_t)1 << 31) return set_err(ctx, MB_EINVAL, "N above 2^31 is not supported");
    cudaStream_t s = (cudaStream_t)stream;
    bool dr, df, du;
    MB_TRY(pointer_kind(ctx, r, &dr));
    MB_TRY(pointer_kind(ctx, f, &df));
    MB_TRY(pointer_kind(ctx, u, &du));
    if (dr != df || dr != du)
        return set_err(ctx, MB_EINVAL, "r, f and u must all be device or all host pointers");
    if (dr) return matvec_device(ctx, r, f, n, a, eta, wall, prec, u, s);
    const size_t bytes = sizeof(double) * 3 * (size_t)n;
    MB_TRY(ensure(ctx, ctx->stage_r, bytes, "host staging"));
    MB_TRY(ensure(ctx, ctx->stage_f, bytes, "host staging"));
    MB_TRY(ensure(ctx, ctx->stage_u, bytes, "host staging"));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->stage_r.ptr, r, bytes, cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->stage_f.ptr, f, bytes, cudaMemcpyHostToDevice, s));
    MB_TRY(matvec_device(ctx, (const double *)ctx->stage_r.ptr, (const double *)ctx->stage_f.ptr,
                         n, a, eta, wall, prec, (double *)ctx->stage_u.ptr, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(u, ctx->stage_u.ptr, bytes, cudaMemcpyDeviceToHost, s));
    MB_TRY(wait_stream(ctx, s, "host-pointer matvec"));
    return MB_OK;
}

mb_status mb_blob_positions(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *q,
                            const double *theta, const int64_t *blob_start, const double *rho,
                            double *r, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_bodies < 0 || n_blobs < 0) return set_err(ctx, MB_EINVAL, "negative size");
    if (n_blobs == 0) return MB_OK;
    if (n_bodies == 0) return set_err(ctx, MB_EINVAL, "blobs without bodies");
    if (!q || !theta || !blob_start || !rho || !r) return set_err(ctx, MB_EINVAL, "null array pointer");
    return blob_positions(ctx, n_bodies, n_blobs, q, theta, blob_start, rho, r,
                          (cudaStream_t)stream);
}

mb_status mb_K_apply(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                     const double *q, const int64_t *blob_start, const double *UO, double *v,
                     void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_bodies < 0 || n_blobs < 0) return set_err(ctx, MB_EINVAL, "negative size");
    if (n_blobs == 0) return MB_OK;
    if (n_bodies == 0) return set_err(ctx, MB_EINVAL, "blobs without bodies");
    if (!r || !q || !blob_start || !UO || !v) return set_err(ctx, MB_EINVAL, "null array pointer");
    launch_K_apply(n_bodies, n_blobs, r, q, blob_start, UO, v, 1.0, 0.0, (cudaStream_t)stream);
    MB_CUDA_TRY(ctx, cudaGetLastError());
    return MB_OK;
}

mb_status mb_KT_apply(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                      const double *q, const int64_t *blob_start, const double *lambda,
                      double *FT, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_bodies < 0 || n_blobs < 0) return set_err(ctx, MB_EINVAL, "negative size");
    if (n_bodies == 0) return MB_OK;
    if (!r || !q || !blob_start || !lambda || !FT) return set_err(ctx, MB_EINVAL, "null array pointer");
    launch_KT_apply(n_bodies, r, q, blob_start, lambda, FT, 1.0, (cudaStream_t)stream);
    MB_CUDA_TRY(ctx, cudaGetLastError());
    return MB_OK;
}

mb_status all_device(mb_context *ctx, std::initializer_list<const void *> ptrs)
{
    for (const void *p : ptrs) {
        bool dev = false;
        MB_TRY(pointer_kind(ctx, p, &dev));
        if (!dev) return set_err(ctx, MB_EINVAL, "arrays must be device pointers");
    }
    return MB_OK;
}

mb_status mb_mobility_eval(mb_context *ctx, const double *x, int64_t n_points, const double *r,
                           const double *f, int64_t n_blobs, double a, double eta, int wall,
                           mb_precision prec, double *u, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_points < 0 || n_blobs < 0) return set_err(ctx, MB_EINVAL, "negative size");
    if (bad_phys(a, eta)) return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (prec != MB_FP64 && prec != MB_FP32_KAHAN)
        return set_err(ctx, MB_EINVAL, "flow evaluation supports MB_FP32_KAHAN and MB_FP64");
    if (n_points == 0) return MB_OK;
    if (!x || !u) return set_err(ctx, MB_EINVAL, "null array pointer");
    if (n_blobs == 0) {
        MB_CUDA_TRY(ctx, cudaMemsetAsync(u, 0, sizeof(double) * 3 * (size_t)n_points,
                                         (cudaStream_t)stream));
        return MB_OK;
    }
    if (!r || !f) return set_err(ctx, MB_EINVAL, "null array pointer");
    MB_TRY(all_device(ctx, {x, r, f, u}));
    return matvec_eval(ctx, x, n_points, r, f, n_blobs, a, eta, wall, prec, u,
                       (cudaStream_t)stream);
}

mb_status mb_render_flow(mb_context *ctx, const double *x, int64_t n_points, const double *r,
                         const double *lambda, int64_t n_blobs, const double *sub_offsets,
                         int n_sub, double a_sub, double eta, int wall, mb_precision prec,
                         double *v, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_points < 0 || n_blobs < 0 || n_sub < 1) return set_err(ctx, MB_EINVAL, "bad sizes");
    if (bad_phys(a_sub, eta)) return set_err(ctx, MB_EINVAL, "a_sub and eta must be positive");
    if (prec != MB_FP64 && prec != MB_FP32_KAHAN)
        return set_err(ctx, MB_EINVAL, "flow rendering supports MB_FP32_KAHAN and MB_FP64");
    if (n_points == 0) return MB_OK;
    if (!x || !v || (n_blobs > 0 && (!r || !lambda || !sub_offsets)))
        return set_err(ctx, MB_EINVAL, "null array pointer");
    if (n_blobs == 0) {
        MB_CUDA_TRY(ctx, cudaMemsetAsync(v, 0, sizeof(double) * 3 * (size_t)n_points,
                                         (cudaStream_t)stream));
        return MB_OK;
    }
    MB_TRY(all_device(ctx, {x, r, lambda, sub_offsets, v}));
    return render_flow(ctx, x, n_points, r, lambda, n_blobs, sub_offsets, n_sub, a_sub, eta, wall,
                       prec, v, (cudaStream_t)stream);
}

mb_status mb_lambda_moments(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                            const double *q, const int64_t *blob_start, const double *lambda,
                            double *S, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_bodies < 0 || n_blobs < 0) return set_err(ctx, MB_EINVAL, "negative size");
    if (n_bodies == 0) return MB_OK;
    if (!r || !q || !blob_start || !lambda || !S) return set_err(ctx, MB_EINVAL, "null array pointer");
    launch_moments(n_bodies, r, q, blob_start, lambda, S, (cudaStream_t)stream);
    MB_CUDA_TRY(ctx, cudaGetLastError());
    return MB_OK;
}

mb_status mb_precond_setup(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *r,
                           const double *q, const int64_t *blob_start, double a, double eta,
                           int wall, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_bodies <= 0 || n_blobs <= 0) return set_err(ctx, MB_EINVAL, "need at least one body");
    if (bad_phys(a, eta)) return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (!r || !q || !blob_start) return set_err(ctx, MB_EINVAL, "null array pointer");
    return precond_setup(ctx, n_bodies, n_blobs, r, q, blob_start, a, eta, wall,
                         (cudaStream_t)stream);
}

mb_status mb_precond_setup_shared(mb_context *ctx, int64_t n_bodies, int64_t n_blobs,
                                  const double *theta, const int64_t *blob_start,
                                  const double *rho, double a, double eta, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_bodies <= 0 || n_blobs <= 0) return set_err(ctx, MB_EINVAL, "need at least one body");
    if (bad_phys(a, eta)) return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (!theta || !blob_start || !rho) return set_err(ctx, MB_EINVAL, "null array pointer");
    return precond_setup_shared(ctx, n_bodies, n_blobs, theta, blob_start, rho, a, eta,
                                (cudaStream_t)stream);
}

mb_status mb_precond_apply(mb_context *ctx, const double *w, const double *g, double *lambda,
                           double *UO, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (!w || !g || !lambda || !UO) return set_err(ctx, MB_EINVAL, "null array pointer");
    return precond_apply_public(ctx, w, g, lambda, UO, (cudaStream_t)stream);
}

mb_status mb_solve_mobility(mb_context *ctx, int64_t n_bodies, int64_t n_blobs, const double *q,
                            const double *theta, const int64_t *blob_start, const double *rho,
                            const double *F, const double *T, const double *slip,
                            const mb_params *params, double *U, double *Omega, double *lambda,
                            mb_info *info, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (!params) return set_err(ctx, MB_EINVAL, "null params");
    if (n_bodies <= 0 || n_blobs <= 0) return set_err(ctx, MB_EINVAL, "need at least one body");
    if (bad_phys(params->a, params->eta))
        return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (!(params->tol > 0.0) || params->maxit < 1 || params->restart < 1)
        return set_err(ctx, MB_EINVAL, "tol > 0, maxit >= 1 and restart >= 1 required");
    if (params->prec != MB_FP64 && params->prec != MB_FP32_KAHAN &&
        params->prec != MB_MIXED_REFINE && params->prec != MB_DF64)
        return set_err(ctx, MB_EINVAL, "unknown precision mode");
    if (params->precond != MB_PRECOND_WALL && params->precond != MB_PRECOND_FREE_SHARED)
        return set_err(ctx, MB_EINVAL, "unknown preconditioner kind");
    if (!q || !theta || !blob_start || !rho || !F || !T || !U || !Omega || !lambda)
        return set_err(ctx, MB_EINVAL, "null array pointer");
    if (n_blobs > (int64_t)1 << 31) return set_err(ctx, MB_EINVAL, "N above 2^31 is not supported");
    return solve_mobility(ctx, n_bodies, n_blobs, q, theta, blob_start, rho, F, T, slip, params, U,
                          Omega, lambda, info, (cudaStream_t)stream);
}

mb_status all_device(mb_context *ctx, std::initializer_list<const void *> ptrs);

mb_status mb_solve_mobility_permeable(mb_context *ctx, int64_t n_bodies, int64_t n_blobs,
                                     const double *q, const double *theta,
                                     const int64_t *blob_start, const double *rho,
                                     const double *F, const double *T, const double *slip,
                                     const double *shift, const mb_params *params, double *U,
                                     double *Omega, double *lambda, mb_info *info, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (!params) return set_err(ctx, MB_EINVAL, "null params");
    if (!shift) return set_err(ctx, MB_EINVAL, "null shift (use mb_solve_mobility)");
    if (params->precond != MB_PRECOND_WALL)
        return set_err(ctx, MB_EINVAL, "permeable bodies use MB_PRECOND_WALL (per-blob shifts "
                                       "make every body's block its own)");
    MB_TRY(all_device(ctx, {shift}));
    if (n_bodies <= 0 || n_blobs <= 0) return set_err(ctx, MB_EINVAL, "need at least one body");
    if (bad_phys(params->a, params->eta))
        return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (!(params->tol > 0.0) || params->maxit < 1 || params->restart < 1)
        return set_err(ctx, MB_EINVAL, "tol > 0, maxit >= 1 and restart >= 1 required");
    if (params->prec != MB_FP64 && params->prec != MB_FP32_KAHAN &&
        params->prec != MB_MIXED_REFINE && params->prec != MB_DF64)
        return set_err(ctx, MB_EINVAL, "unknown precision mode");
    if (!q || !theta || !blob_start || !rho || !F || !T || !U || !Omega || !lambda)
        return set_err(ctx, MB_EINVAL, "null array pointer");
    if (n_blobs > (int64_t)1 << 31) return set_err(ctx, MB_EINVAL, "N above 2^31 is not supported");
    return solve_mobility(ctx, n_bodies, n_blobs, q, theta, blob_start, rho, F, T, slip, params, U,
                          Omega, lambda, info, (cudaStream_t)stream, shift);
}

mb_status mb_solve_resistance(mb_context *ctx, int64_t n_bodies, int64_t n_blobs,
                              const double *q, const double *theta, const int64_t *blob_start,
                              const double *rho, const double *U, const double *Omega,
                              const double *slip, const mb_params *params, double *F, double *T,
                              double *lambda, mb_info *info, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (!params) return set_err(ctx, MB_EINVAL, "null params");
    if (n_bodies <= 0 || n_blobs <= 0) return set_err(ctx, MB_EINVAL, "need at least one body");
    if (bad_phys(params->a, params->eta))
        return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (!(params->tol > 0.0) || params->maxit < 1 || params->restart < 1)
        return set_err(ctx, MB_EINVAL, "tol > 0, maxit >= 1 and restart >= 1 required");
    if (params->prec != MB_FP64 && params->prec != MB_FP32_KAHAN &&
        params->prec != MB_MIXED_REFINE && params->prec != MB_DF64)
        return set_err(ctx, MB_EINVAL, "unknown precision mode");
    if (params->precond != MB_PRECOND_WALL && params->precond != MB_PRECOND_FREE_SHARED)
        return set_err(ctx, MB_EINVAL, "unknown preconditioner kind");
    if (!q || !theta || !blob_start || !rho || !U || !Omega || !F || !T || !lambda)
        return set_err(ctx, MB_EINVAL, "null array pointer");
    if (n_blobs > (int64_t)1 << 31) return set_err(ctx, MB_EINVAL, "N above 2^31 is not supported");
    return solve_resistance(ctx, n_bodies, n_blobs, q, theta, blob_start, rho, U, Omega, slip,
                            params, F, T, lambda, info, (cudaStream_t)stream);
}

mb_status mb_solve_batch(mb_context *ctx, int n_problems, const mb_problem *problems,
                         const mb_params *params, mb_info *infos, void *stream)
{
    MB_TRY(check_ctx(ctx));
    if (n_problems < 0 || (n_problems > 0 && !problems) || !params)
        return set_err(ctx, MB_EINVAL, "bad problem list or null params");
    if (n_problems == 0) return MB_OK;
    if (bad_phys(params->a, params->eta))
        return set_err(ctx, MB_EINVAL, "a and eta must be positive and finite");
    if (!(params->tol > 0.0) || params->maxit < 1 || params->restart < 1)
        return set_err(ctx, MB_EINVAL, "tol > 0, maxit >= 1 and restart >= 1 required");
    if (params->prec != MB_FP64 && params->prec != MB_FP32_KAHAN &&
        params->prec != MB_MIXED_REFINE && params->prec != MB_DF64)
        return set_err(ctx, MB_EINVAL, "unknown precision mode");
    if (params->precond != MB_PRECOND_WALL)
        return set_err(ctx, MB_EINVAL, "the batched engine uses MB_PRECOND_WALL only");
    int64_t n_tot = 0;
    for (int p = 0; p < n_problems; ++p) {
        const mb_problem &P = problems[p];
        if (P.n_bodies <= 0 || P.n_blobs <= 0)
            return set_err(ctx, MB_EINVAL, "problem %d: needs at least one body and one blob", p);
        if (!P.q || !P.theta || !P.blob_start || !P.rho || !P.F || !P.T || !P.U || !P.Omega ||
            !P.lambda)
            return set_err(ctx, MB_EINVAL, "problem %d: null array pointer", p);
        n_tot += P.n_blobs;
    }
    if (n_tot > (int64_t)1 << 31) return set_err(ctx, MB_EINVAL, "total N above 2^31");
    return solve_batch(ctx, n_problems, problems, params, infos, (cudaStream_t)stream);
}

}  // extern "C"
