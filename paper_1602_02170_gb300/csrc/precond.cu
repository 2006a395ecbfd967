// Block-diagonal indefinite preconditioner (Section 2.2.2).
//
// For each body p with n = 3 n_p rows, Eq. M_tilde_block_diag keeps only its
// own blob mobility block M_p = M^(pp) (with the wall).  Applying Eq.
// indef_block_P means solving, body by body,
//     M_p lambda_p - K_p U_p = w_p,    -K_p^T lambda_p = g_p,
// whose solution is U_p = -N_p (g_p + Q_p^T w_p), lambda_p = M_p^-1 w_p + Q_p U_p
// with Q_p = M_p^-1 K_p and N_p = (K_p^T M_p^-1 K_p)^-1, the body mobility of
// body p alone.  The setup kernel (one CTA per body) assembles M_p in FP64,
// factors it by Cholesky, forms M_p^-1 by column solves, Q_p, the 6 x 6
// Schur complement and N_p, and stores the explicit (n+6) x (n+6) inverse
//     P_p^-1 = [[M_p^-1 - Q_p N_p Q_p^T, -Q_p N_p], [-N_p Q_p^T, -N_p]],
// so that one application is one batched FP64 GEMV per body.
#include <algorithm>
#include <vector>

#include "mb_internal.cuh"
#include "rpy_wall.cuh"

namespace mb {
namespace {

constexpr int kSetupThreads = 256;
constexpr int kSmemMaxRows = 160;   // n = 3 n_p rows held in shared memory up to this

// Shared-memory layout of the setup kernel: [L (n*n, only if in smem) | Q (n*6) | QN (n*6) | S (36) | N (36)]
template <bool WALL, bool L_SMEM>
__global__ void __launch_bounds__(kSetupThreads) precond_setup_kernel(
    int64_t nb, const double *__restrict__ r, const double *__restrict__ q,
    const int64_t *__restrict__ start, const int64_t *__restrict__ poff, PairConsts<double> k,
    double scale, double *__restrict__ P, double *__restrict__ scratch, int64_t scratch_stride,
    int *__restrict__ flag, int flag_slot)
{
    extern __shared__ double sm[];
    for (int64_t p = blockIdx.x; p < nb; p += gridDim.x) {
        const int64_t b0 = start[p];
        const int np = (int)(start[p + 1] - b0);
        const int n = 3 * np;
        const int m = n + 6;
        double *L = L_SMEM ? sm : scratch + blockIdx.x * scratch_stride;
        double *Q = L_SMEM ? sm + (size_t)n * n : sm;
        double *QN = Q + 6 * n;
        double *S = QN + 6 * n;
        double *Nm = S + 36;
        __shared__ int bad;
        double *Pp = P + poff[p];
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        if (threadIdx.x == 0) bad = 0;

        // 1. assemble M_p (full square, FP64)
        for (int e = threadIdx.x; e < np * np; e += blockDim.x) {
            const int bi = e / np, bj = e % np;
            double blk[9];
            block_f64<WALL>(r + 3 * (b0 + bi), r + 3 * (b0 + bj), k, blk);
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be)
                    L[(3 * bi + al) * n + 3 * bj + be] = scale * blk[3 * al + be];
        }
        __syncthreads();

        // 2. right-looking Cholesky, lower triangle in place
        for (int c = 0; c < n; ++c) {
            if (threadIdx.x == 0) {
                const double d = L[c * n + c];
                if (!(d > 0.0)) bad = 1;
                L[c * n + c] = sqrt(fabs(d));
            }
            __syncthreads();
            if (bad) break;
            const double dinv = 1.0 / L[c * n + c];
            for (int i = c + 1 + threadIdx.x; i < n; i += blockDim.x) L[i * n + c] *= dinv;
            __syncthreads();
            const int w = n - c - 1;
            for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
                const int i = c + 1 + e / w, j = c + 1 + e % w;
                if (j <= i) L[i * n + j] -= L[i * n + c] * L[j * n + c];
            }
            __syncthreads();
        }
        if (bad) {
            if (threadIdx.x == 0) {
                if (flag_slot >= 0) flag[flag_slot] = 2;
                else atomicMin(flag, (int)p);
            }
            __syncthreads();
            continue;
        }

        // 3. X = M_p^-1 by column solves L y = e_c, L^T x = y; column c lives in
        //    P_p[:, c] (row stride m), one thread per column
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            for (int i = 0; i < c; ++i) Pp[(size_t)i * m + c] = 0.0;
            for (int i = c; i < n; ++i) {
                double acc = (i == c) ? 1.0 : 0.0;
                for (int kk = c; kk < i; ++kk) acc -= L[i * n + kk] * Pp[(size_t)kk * m + c];
                Pp[(size_t)i * m + c] = acc / L[i * n + i];
            }
            for (int i = n - 1; i >= 0; --i) {
                double acc = Pp[(size_t)i * m + c];
                for (int kk = i + 1; kk < n; ++kk) acc -= L[kk * n + i] * Pp[(size_t)kk * m + c];
                Pp[(size_t)i * m + c] = acc / L[i * n + i];
            }
        }
        __syncthreads();

        // 4. Q = X K_p (n x 6); K_p row block of blob i is [I, -[d_i]_x]
        for (int e = threadIdx.x; e < 6 * n; e += blockDim.x) {
            const int row = e / 6, col = e % 6;
            double acc = 0.0;
            for (int i = 0; i < np; ++i) {
                const double *x = Pp + (size_t)row * m + 3 * i;
                if (col < 3) {
                    acc += x[col];
                } else {
                    const double dx = r[3 * (b0 + i)] - qx, dy = r[3 * (b0 + i) + 1] - qy,
                                 dz = r[3 * (b0 + i) + 2] - qz;
                    // column (col-3) of -[d]_x
                    if (col == 3) acc += -dz * x[1] + dy * x[2];
                    else if (col == 4) acc += dz * x[0] - dx * x[2];
                    else acc += -dy * x[0] + dx * x[1];
                }
            }
            Q[row * 6 + col] = acc;
        }
        __syncthreads();

        // 5. S = K_p^T Q (6 x 6)
        if (threadIdx.x < 36) {
            const int a = threadIdx.x / 6, b = threadIdx.x % 6;
            double acc = 0.0;
            for (int i = 0; i < np; ++i) {
                const double *qr = Q + 3 * i * 6;  // rows 3i..3i+2
                if (a < 3) {
                    acc += qr[a * 6 + b];
                } else {
                    const double dx = r[3 * (b0 + i)] - qx, dy = r[3 * (b0 + i) + 1] - qy,
                                 dz = r[3 * (b0 + i) + 2] - qz;
                    // row (a-3) of (-[d]_x)^T = [d]_x
                    if (a == 3) acc += -dz * qr[1 * 6 + b] + dy * qr[2 * 6 + b];
                    else if (a == 4) acc += dz * qr[0 * 6 + b] - dx * qr[2 * 6 + b];
                    else acc += -dy * qr[0 * 6 + b] + dx * qr[1 * 6 + b];
                }
            }
            S[a * 6 + b] = acc;
        }
        __syncthreads();

        // 6. N = S^-1 by Gauss-Jordan on the symmetrised S (one thread)
        if (threadIdx.x == 0) {
            double A[6][12];
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) {
                    A[a][b] = 0.5 * (S[a * 6 + b] + S[b * 6 + a]);
                    A[a][6 + b] = (a == b) ? 1.0 : 0.0;
                }
            for (int c = 0; c < 6 && !bad; ++c) {
                const double d = A[c][c];
                if (!(d > 0.0)) { bad = 1; break; }
                for (int b = 0; b < 12; ++b) A[c][b] /= d;
                for (int a = 0; a < 6; ++a)
                    if (a != c) {
                        const double f = A[a][c];
                        for (int b = 0; b < 12; ++b) A[a][b] -= f * A[c][b];
                    }
            }
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b) Nm[a * 6 + b] = A[a][6 + b];
        }
        __syncthreads();
        if (bad) {
            if (threadIdx.x == 0) {
                if (flag_slot >= 0) flag[flag_slot] = 2;
                else atomicMin(flag, (int)p);
            }
            __syncthreads();
            continue;
        }

        // 7. QN = Q N
        for (int e = threadIdx.x; e < 6 * n; e += blockDim.x) {
            const int row = e / 6, col = e % 6;
            double acc = 0.0;
#pragma unroll
            for (int kk = 0; kk < 6; ++kk) acc += Q[row * 6 + kk] * Nm[kk * 6 + col];
            QN[row * 6 + col] = acc;
        }
        __syncthreads();

        // 8. P_p^-1 = [[X - QN Q^T, -QN], [-QN^T, -N]]
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = e / m, j = e % m;
            double v;
            if (i < n && j < n) {
                double acc = 0.0;
#pragma unroll
                for (int kk = 0; kk < 6; ++kk) acc += QN[i * 6 + kk] * Q[j * 6 + kk];
                v = Pp[(size_t)i * m + j] - acc;
            } else if (i < n) {
                v = -QN[i * 6 + (j - n)];
            } else if (j < n) {
                v = -QN[j * 6 + (i - n)];
            } else {
                v = -Nm[(i - n) * 6 + (j - n)];
            }
            Pp[(size_t)i * m + j] = v;
        }
        __syncthreads();
    }
}

// z_p = P_p^-1 [w_p; g_p] for every body; one CTA per body (grid-stride),
// one warp per output row, lanes across the row.
__global__ void __launch_bounds__(256) precond_apply_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    const double *__restrict__ P, const double *__restrict__ w, const double *__restrict__ g,
    double *__restrict__ lam, double *__restrict__ UO)
{
    extern __shared__ double xs[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t p = blockIdx.x; p < nb; p += gridDim.x) {
        const int64_t b0 = start[p];
        const int n = 3 * (int)(start[p + 1] - b0);
        const int m = n + 6;
        __syncthreads();
        for (int e = threadIdx.x; e < m; e += blockDim.x)
            xs[e] = e < n ? w[3 * b0 + e] : g[6 * p + (e - n)];
        __syncthreads();
        const double *Pp = P + poff[p];
        for (int row = warp; row < m; row += nw) {
            const double *pr = Pp + (size_t)row * m;
            double acc = 0.0;
            for (int c = lane; c < m; c += 32) acc += pr[c] * xs[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                if (row < n) lam[3 * b0 + row] = acc;
                else UO[6 * p + (row - n)] = acc;
            }
        }
    }
}

}  // namespace

mb_status precond_setup(mb_context *ctx, int64_t nb, int64_t n, const double *r,
                        const double *q, const int64_t *blob_start, double a, double eta,
                        int wall, cudaStream_t s)
{
    // body sizes on the host
    std::vector<int64_t> hstart(nb + 1);
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(hstart.data(), blob_start, sizeof(int64_t) * (nb + 1),
                                     cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hstart[0] != 0 || hstart[nb] != n)
        return set_err(ctx, MB_EINVAL, "blob_start[0] must be 0 and blob_start[n_b] = N");
    std::vector<int64_t> off(nb + 1);
    off[0] = 0;
    int max_np = 0;
    for (int64_t p = 0; p < nb; ++p) {
        const int64_t np = hstart[p + 1] - hstart[p];
        if (np < 1) return set_err(ctx, MB_EINVAL, "body %lld has no blobs", (long long)p);
        max_np = std::max<int>(max_np, (int)np);
        off[p + 1] = off[p] + (3 * np + 6) * (3 * np + 6);
    }
    MB_TRY(ensure(ctx, ctx->pinv, sizeof(double) * off[nb], "preconditioner"));
    MB_TRY(ensure(ctx, ctx->pinv_off, sizeof(int64_t) * (nb + 1), "preconditioner"));
    MB_TRY(ensure(ctx, ctx->blob_start_copy, sizeof(int64_t) * (nb + 1), "preconditioner"));
    MB_TRY(ensure(ctx, ctx->flag, sizeof(int) * 4, "flags"));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinv_off.ptr, off.data(), sizeof(int64_t) * (nb + 1),
                                     cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->blob_start_copy.ptr, hstart.data(),
                                     sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    const int big = 0x7fffffff;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->flag.ptr, &big, sizeof(int), cudaMemcpyHostToDevice, s));

    const int nmax = 3 * max_np;
    const bool lsmem = nmax <= kSmemMaxRows;
    const size_t small = sizeof(double) * (12 * (size_t)nmax + 72);
    const size_t smem = small + (lsmem ? sizeof(double) * (size_t)nmax * nmax : 0);
    const PairConsts<double> k = PairConsts<double>::make(a);
    const double scale = 1.0 / (6.0 * 3.14159265358979323846 * eta * a);
    int grid = (int)std::min<int64_t>(nb, 4 * (int64_t)ctx->sm_count);
    double *scratch = nullptr;
    int64_t stride = 0;
    if (!lsmem) {
        grid = (int)std::min<int64_t>(nb, ctx->sm_count);
        stride = (int64_t)nmax * nmax;
        MB_TRY(ensure(ctx, ctx->sol_dots, sizeof(double) * stride * grid, "Cholesky scratch"));
        scratch = (double *)ctx->sol_dots.ptr;
    }
    auto launch = [&](auto kern) -> mb_status {
        MB_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        kern<<<grid, kSetupThreads, smem, s>>>(nb, r, q, (const int64_t *)ctx->blob_start_copy.ptr,
                                               (const int64_t *)ctx->pinv_off.ptr, k, scale,
                                               (double *)ctx->pinv.ptr, scratch, stride,
                                               (int *)ctx->flag.ptr, -1);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    };
    if (wall) {
        MB_TRY(lsmem ? launch(precond_setup_kernel<true, true>)
                     : launch(precond_setup_kernel<true, false>));
    } else {
        MB_TRY(lsmem ? launch(precond_setup_kernel<false, true>)
                     : launch(precond_setup_kernel<false, false>));
    }
    int first_bad = big;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(&first_bad, ctx->flag.ptr, sizeof(int),
                                     cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    ctx->pc_nb = nb;
    ctx->pc_n = n;
    ctx->pc_max_np = max_np;
    if (first_bad != big) {
        ctx->pc_nb = 0;
        return set_err(ctx, MB_ESINGULAR,
                       "body %d: mobility block or its Schur complement is not positive definite",
                       first_bad);
    }
    return MB_OK;
}

mb_status precond_setup_range(mb_context *ctx, int64_t nb, const double *r, const double *q,
                              const int64_t *start, const int64_t *poff, double *P, int max_np,
                              double a, double eta, int wall, int *flags, int flag_slot,
                              cudaStream_t s)
{
    const int nmax = 3 * max_np;
    const bool lsmem = nmax <= kSmemMaxRows;
    const size_t small = sizeof(double) * (12 * (size_t)nmax + 72);
    const size_t smem = small + (lsmem ? sizeof(double) * (size_t)nmax * nmax : 0);
    const PairConsts<double> k = PairConsts<double>::make(a);
    const double scale = 1.0 / (6.0 * 3.14159265358979323846 * eta * a);
    int grid = (int)std::min<int64_t>(nb, 4 * (int64_t)ctx->sm_count);
    double *scratch = nullptr;
    int64_t stride = 0;
    if (!lsmem) {
        grid = (int)std::min<int64_t>(nb, ctx->sm_count);
        stride = (int64_t)nmax * nmax;
        MB_TRY(ensure(ctx, ctx->sol_dots, sizeof(double) * stride * grid, "Cholesky scratch"));
        scratch = (double *)ctx->sol_dots.ptr;
    }
    auto launch = [&](auto kern) -> mb_status {
        MB_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        kern<<<grid, kSetupThreads, smem, s>>>(nb, r, q, start, poff, k, scale, P, scratch, stride,
                                               flags, flag_slot);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    };
    if (wall)
        return lsmem ? launch(precond_setup_kernel<true, true>)
                     : launch(precond_setup_kernel<true, false>);
    return lsmem ? launch(precond_setup_kernel<false, true>)
                 : launch(precond_setup_kernel<false, false>);
}

static void precond_apply_impl(mb_context *ctx, const double *w, const double *g, double *lam,
                               double *UO, cudaStream_t s)
{
    const int m = 3 * ctx->pc_max_np + 6;
    const int grid = (int)std::min<int64_t>(ctx->pc_nb, 8 * (int64_t)ctx->sm_count);
    precond_apply_kernel<<<grid, 256, sizeof(double) * m, s>>>(
        ctx->pc_nb, (const int64_t *)ctx->blob_start_copy.ptr, (const int64_t *)ctx->pinv_off.ptr,
        (const double *)ctx->pinv.ptr, w, g, lam, UO);
    count_launch();
}

void precond_apply_packed(mb_context *ctx, const double *v, double *z, cudaStream_t s)
{
    const int64_t n3 = 3 * ctx->pc_n;
    precond_apply_impl(ctx, v, v + n3, z, z + n3, s);
}

mb_status precond_apply_public(mb_context *ctx, const double *w, const double *g, double *lam,
                               double *UO, cudaStream_t s)
{
    if (ctx->pc_nb == 0) return set_err(ctx, MB_EINVAL, "no preconditioner has been set up");
    if (3 * ctx->pc_max_np + 6 > 6000)
        return set_err(ctx, MB_EINVAL, "body too large for the preconditioner apply");
    precond_apply_impl(ctx, w, g, lam, UO, s);
    MB_CUDA_TRY(ctx, cudaGetLastError());
    return MB_OK;
}

}  // namespace mb
