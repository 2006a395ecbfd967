// Rigid-body geometry and kinematics on the blobs.
//   blob build:  r_i = q_p + R(theta_p) rho_i                    (Section 2.1)
//   K:           v_i = U_p + Omega_p x (r_i - q_p)               (Eq. noslip_rigid)
//   K^T:         (sum_i lambda_i, sum_i (r_i - q_p) x lambda_i)  (Eq. rigidSystem)
// One thread per blob for the gathers (the body is found by binary search in
// the CSR offsets), one warp per body for the segmented reduction of K^T.
#include <algorithm>

#include "mb_internal.cuh"

namespace mb {
namespace {

__global__ void blob_positions_kernel(int64_t nb, int64_t n, const double *__restrict__ q,
                                      const double *__restrict__ theta,
                                      const int64_t *__restrict__ start,
                                      const double *__restrict__ rho, double *__restrict__ r)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = body_of(start, nb, i);
        double s = theta[4 * p], x = theta[4 * p + 1], y = theta[4 * p + 2], z = theta[4 * p + 3];
        const double inv = rsqrt(s * s + x * x + y * y + z * z);
        s *= inv; x *= inv; y *= inv; z *= inv;
        const double a = rho[3 * i], b = rho[3 * i + 1], c = rho[3 * i + 2];
        // R = (s^2 - v.v) I + 2 v v^T + 2 s [v]_x, applied to (a, b, c)
        const double d = s * s - (x * x + y * y + z * z);
        const double vr = x * a + y * b + z * c;
        r[3 * i + 0] = q[3 * p + 0] + d * a + 2.0 * x * vr + 2.0 * s * (y * c - z * b);
        r[3 * i + 1] = q[3 * p + 1] + d * b + 2.0 * y * vr + 2.0 * s * (z * a - x * c);
        r[3 * i + 2] = q[3 * p + 2] + d * c + 2.0 * z * vr + 2.0 * s * (x * b - y * a);
    }
}

__global__ void K_apply_kernel(int64_t nb, int64_t n, const double *__restrict__ r,
                               const double *__restrict__ q, const int64_t *__restrict__ start,
                               const double *__restrict__ UO, double *__restrict__ v, double alpha,
                               double beta)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = body_of(start, nb, i);
        const double dx = r[3 * i] - q[3 * p], dy = r[3 * i + 1] - q[3 * p + 1],
                     dz = r[3 * i + 2] - q[3 * p + 2];
        const double *u = UO + 6 * p;
        const double vx = u[0] + (u[4] * dz - u[5] * dy);
        const double vy = u[1] + (u[5] * dx - u[3] * dz);
        const double vz = u[2] + (u[3] * dy - u[4] * dx);
        if (beta == 0.0) {
            v[3 * i] = alpha * vx;
            v[3 * i + 1] = alpha * vy;
            v[3 * i + 2] = alpha * vz;
        } else {
            v[3 * i] = alpha * vx + beta * v[3 * i];
            v[3 * i + 1] = alpha * vy + beta * v[3 * i + 1];
            v[3 * i + 2] = alpha * vz + beta * v[3 * i + 2];
        }
    }
}

__global__ void KT_apply_kernel(int64_t nb, const double *__restrict__ r, const double *__restrict__ q,
                                const int64_t *__restrict__ start, const double *__restrict__ lam,
                                double *__restrict__ FT, double alpha)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < nb;
         p += warps) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        for (int64_t i = start[p] + lane; i < start[p + 1]; i += 32) {
            const double lx = lam[3 * i], ly = lam[3 * i + 1], lz = lam[3 * i + 2];
            const double dx = r[3 * i] - qx, dy = r[3 * i + 1] - qy, dz = r[3 * i + 2] - qz;
            acc[0] += lx;
            acc[1] += ly;
            acc[2] += lz;
            acc[3] += dy * lz - dz * ly;
            acc[4] += dz * lx - dx * lz;
            acc[5] += dx * ly - dy * lx;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        }
        if (lane < 6) {
            double v = acc[0];
#pragma unroll
            for (int c = 1; c < 6; ++c)
                if (lane == c) v = acc[c];
            FT[6 * p + lane] = alpha * v;
        }
    }
}

// The same sum with one CTA per body, for few bodies (the warp-per-body form
// would leave most SMs idle and run each body's blobs serially in one warp).
constexpr int64_t kKTBlockBodies = 256;

__global__ void __launch_bounds__(256) KT_apply_block_kernel(
    int64_t nb, const double *__restrict__ r, const double *__restrict__ q,
    const int64_t *__restrict__ start, const double *__restrict__ lam, double *__restrict__ FT,
    double alpha)
{
    __shared__ double red[8][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t p = blockIdx.x; p < nb; p += gridDim.x) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        for (int64_t i = start[p] + threadIdx.x; i < start[p + 1]; i += blockDim.x) {
            const double lx = lam[3 * i], ly = lam[3 * i + 1], lz = lam[3 * i + 2];
            const double dx = r[3 * i] - qx, dy = r[3 * i + 1] - qy, dz = r[3 * i + 2] - qz;
            acc[0] += lx;
            acc[1] += ly;
            acc[2] += lz;
            acc[3] += dy * lz - dz * ly;
            acc[4] += dz * lx - dx * lz;
            acc[5] += dx * ly - dy * lx;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        }
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) red[warp][c] = acc[c];
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double v = 0.0;
            for (int w8 = 0; w8 < 8; ++w8) v += red[w8][threadIdx.x];
            FT[6 * p + threadIdx.x] = alpha * v;
        }
    }
}

static_assert(kSaddleRowsMaxBodies == kKTBlockBodies,
              "saddle_rows_kernel reduces K^T lambda with one CTA per body");

// The saddle operator's rows around M lambda in one launch (Eq. saddle_M),
// from the pair kernel's chunk partials; x = [lambda; U].  Blocks below
// blob_blocks take blobs, one thread per blob:
//   y_i = scale * sum_s partial[s][i] - (K U)_i
// (the sums of reduce_partials_kernel, then K_apply_kernel with alpha = -1,
// beta = 1); the other blocks take bodies, one CTA per body:
//   y_(3N + 6p + c) = -(K^T lambda)_p,c
// (the reduction of KT_apply_block_kernel).  All threads of a block take the
// same branch, so the barriers of the body branch are uniform.  Blocks are
// small (kSaddleThreads): the per-thread work is a short serial chain of FP64
// instructions, which issue slowly on this chip, so spreading the warps over
// more SMs shortens the launch; for bodies of up to 64 blobs the body sums
// round as with one CTA of 256 threads.
constexpr int kSaddleThreads = 64;

__global__ void __launch_bounds__(kSaddleThreads) saddle_rows_kernel(
    const double *__restrict__ partial, int S, double scale, int64_t n, int64_t nb,
    const double *__restrict__ r, const double *__restrict__ q, const int64_t *__restrict__ start,
    const double *__restrict__ x, double *__restrict__ y, int blob_blocks)
{
    const int64_t m = 3 * n;
    if ((int)blockIdx.x < blob_blocks) {
        const double *UO = x + m;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)blob_blocks * blockDim.x) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int sc = 0; sc < S; ++sc) {
                const double *ps = partial + sc * m + 3 * i;
                acc[0] += ps[0];
                acc[1] += ps[1];
                acc[2] += ps[2];
            }
            const int64_t p = body_of(start, nb, i);
            const double dx = r[3 * i] - q[3 * p], dy = r[3 * i + 1] - q[3 * p + 1],
                         dz = r[3 * i + 2] - q[3 * p + 2];
            const double *u = UO + 6 * p;
            const double vx = u[0] + (u[4] * dz - u[5] * dy);
            const double vy = u[1] + (u[5] * dx - u[3] * dz);
            const double vz = u[2] + (u[3] * dy - u[4] * dx);
            // rounded as the two-kernel sequence: u = scale * acc, then u - v
            y[3 * i] = __dsub_rn(__dmul_rn(scale, acc[0]), vx);
            y[3 * i + 1] = __dsub_rn(__dmul_rn(scale, acc[1]), vy);
            y[3 * i + 2] = __dsub_rn(__dmul_rn(scale, acc[2]), vz);
        }
        return;
    }
    constexpr int kWarps = kSaddleThreads / 32;
    __shared__ double red[kWarps][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int body_blocks = (int)gridDim.x - blob_blocks;
    for (int64_t p = (int)blockIdx.x - blob_blocks; p < nb; p += body_blocks) {
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        for (int64_t i = start[p] + threadIdx.x; i < start[p + 1]; i += blockDim.x) {
            const double lx = x[3 * i], ly = x[3 * i + 1], lz = x[3 * i + 2];
            const double dx = r[3 * i] - qx, dy = r[3 * i + 1] - qy, dz = r[3 * i + 2] - qz;
            acc[0] += lx;
            acc[1] += ly;
            acc[2] += lz;
            acc[3] += dy * lz - dz * ly;
            acc[4] += dz * lx - dx * lz;
            acc[5] += dx * ly - dy * lx;
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        }
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) red[warp][c] = acc[c];
        }
        __syncthreads();
        if (threadIdx.x < 6) {
            double v = 0.0;
            for (int w8 = 0; w8 < kWarps; ++w8) v += red[w8][threadIdx.x];
            y[m + 6 * p + threadIdx.x] = -v;
        }
    }
}

int grid_for(int64_t work, int threads)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, threads), 4096));
}

}  // namespace

mb_status blob_positions(mb_context *ctx, int64_t nb, int64_t n, const double *q,
                         const double *theta, const int64_t *blob_start, const double *rho,
                         double *r, cudaStream_t s)
{
    if (n == 0) return MB_OK;
    blob_positions_kernel<<<grid_for(n, 256), 256, 0, s>>>(nb, n, q, theta, blob_start, rho, r);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    return MB_OK;
}

void launch_K_apply(int64_t nb, int64_t n, const double *r, const double *q,
                    const int64_t *blob_start, const double *UO, double *v, double alpha,
                    double beta, cudaStream_t s)
{
    if (n == 0) return;
    K_apply_kernel<<<grid_for(n, 256), 256, 0, s>>>(nb, n, r, q, blob_start, UO, v, alpha, beta);
    count_launch();
}

void launch_saddle_rows(const MatvecPartials &mp, int64_t n, int64_t nb, const double *r,
                        const double *q, const int64_t *blob_start, const double *x, double *y,
                        cudaStream_t s)
{
    const int blob_blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, kSaddleThreads), 4096));
    saddle_rows_kernel<<<blob_blocks + (int)nb, kSaddleThreads, 0, s>>>(
        mp.partial, mp.S, mp.scale, n, nb, r, q, blob_start, x, y, blob_blocks);
    count_launch();
}

// S_p[a][b] = sum_{i in p} lambda_i,a (r_i - q_p)_b: the first moment of the
// blob forces, whose symmetric traceless part is the body's stresslet
// (Section 4.1).  One warp per body.
__global__ void moments_kernel(int64_t nb, const double *__restrict__ r,
                               const double *__restrict__ q, const int64_t *__restrict__ start,
                               const double *__restrict__ lam, double *__restrict__ S)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < nb;
         p += warps) {
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        for (int64_t i = start[p] + lane; i < start[p + 1]; i += 32) {
            const double d[3] = {r[3 * i] - qx, r[3 * i + 1] - qy, r[3 * i + 2] - qz};
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be) acc[3 * al + be] += lam[3 * i + al] * d[be];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        }
        if (lane < 9) {
            double v = acc[0];
#pragma unroll
            for (int c = 1; c < 9; ++c)
                if (lane == c) v = acc[c];
            S[9 * p + lane] = v;
        }
    }
}

void launch_moments(int64_t nb, const double *r, const double *q, const int64_t *blob_start,
                    const double *lambda, double *S, cudaStream_t s)
{
    if (nb == 0) return;
    moments_kernel<<<grid_for(nb * 32, 256), 256, 0, s>>>(nb, r, q, blob_start, lambda, S);
    count_launch();
}

void launch_KT_apply(int64_t nb, const double *r, const double *q, const int64_t *blob_start,
                     const double *lambda, double *FT, double alpha, cudaStream_t s)
{
    if (nb == 0) return;
    if (nb <= kKTBlockBodies)
        KT_apply_block_kernel<<<(int)nb, 256, 0, s>>>(nb, r, q, blob_start, lambda, FT, alpha);
    else
        KT_apply_kernel<<<grid_for(nb * 32, 256), 256, 0, s>>>(nb, r, q, blob_start, lambda, FT,
                                                               alpha);
    count_launch();
}

}  // namespace mb
