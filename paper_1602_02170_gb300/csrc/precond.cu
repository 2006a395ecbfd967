// Block-diagonal indefinite preconditioner (Section 2.2.2).
//
// For each body p with n = 3 n_p rows, Eq. M_tilde_block_diag keeps only its
// own blob mobility block M_p = M^(pp) (with the wall).  Applying Eq.
// indef_block_P means solving, body by body,
//     M_p lambda_p - K_p U_p = w_p,    -K_p^T lambda_p = g_p,
// whose solution is U_p = -N_p (g_p + Q_p^T w_p), lambda_p = M_p^-1 w_p + Q_p U_p
// with Q_p = M_p^-1 K_p and N_p = (K_p^T M_p^-1 K_p)^-1, the body mobility of
// body p alone.  The setup kernel (one CTA per body) assembles M_p in FP64,
// factors it by Cholesky M_p = L L^T, inverts the factor (W = L^-1, kept
// transposed in the free upper triangle), forms M_p^-1 = W^T W, Q_p, the 6 x 6
// Schur complement and N_p, and stores the explicit (n+6) x (n+6) inverse
//     P_p^-1 = [[M_p^-1 - Q_p N_p Q_p^T, -Q_p N_p], [-N_p Q_p^T, -N_p]],
// so that one application is one batched FP64 GEMV per body.
#include <algorithm>
#include <cstring>
#include <unordered_map>
#include <vector>

#include <cooperative_groups.h>

#include "df32.cuh"
#include "mb_internal.cuh"
#include "rpy_wall.cuh"

namespace mb {
namespace {

#ifndef MB_SETUP_SCRATCH_MB
#define MB_SETUP_SCRATCH_MB 256  // scratch of one group of bodies in the split setup
#endif
constexpr int kSetupThreads = 256;
constexpr int kSmemMaxRows = 160;   // n = 3 n_p rows held in shared memory up to this

// The pivot test and 1 / sqrt(d) of the factorisations, with few FP64
// instructions: an FP64 warp instruction (compares and conversions included)
// issues only about once per 76 cycles on each SM sub-partition of this chip,
// and the pivots sit on the factorisation's serial chain.
//   pivot_ok: d > 0 and finite, from the bit pattern (integer compares).
//   pivot_rsqrt: an FP32 estimate from d's truncated bits (integer
//     operations), one FP32 Newton step, back to FP64 through the bit pattern
//     (exact), then one FP64 Newton step y + (y / 2)(1 - d y^2) in three FP64
//     instructions: about 2e-14 relative (quadratic convergence from the
//     FP32 estimate's ~2^-23).  Exponents outside 2^-100 .. 2^100 take
//     1 / sqrt(d).
__device__ __forceinline__ bool pivot_ok(double d)
{
    const long long b = __double_as_longlong(d);
    return b > 0 && b < 0x7ff0000000000000LL;
}

// FP64 number with the bits of a positive normal FP32 number (exact)
__device__ __forceinline__ double f32_to_f64_bits(float y)
{
    const unsigned yb = __float_as_uint(y);
    return __hiloint2double((int)((((yb >> 23) + 896u) << 20) | ((yb & 0x7fffffu) >> 3)),
                            (int)((yb & 7u) << 29));
}

// FP32 number with the exponent of d (2^-100 .. 2^100) and the top 23 bits
// of its mantissa
__device__ __forceinline__ float f64_to_f32_trunc(double d)
{
    const int hi = __double2hiint(d);
    const unsigned lo = (unsigned)__double2loint(d);
    return __int_as_float(((hi - (896 << 20)) << 3) | (int)(lo >> 29));
}

__device__ __forceinline__ bool f32_range(double d)
{
    const int e = (__double2hiint(d) >> 20) & 0x7ff;
    return e >= 1023 - 100 && e <= 1023 + 100;
}

// 1 / d for positive d the same way: FP32 estimate with one FP32 Newton
// step, then y + y (1 - d y) in two FP64 instructions (~1e-14 relative).
__device__ __forceinline__ double pivot_rcp(double d)
{
    if (!f32_range(d)) return 1.0 / d;
    const float f = f64_to_f32_trunc(d);
    float y = __fdividef(1.0f, f);
    y = y * (2.0f - f * y);
    const double yd = f32_to_f64_bits(y);
    return fma(yd, fma(-d, yd, 1.0), yd);
}

__device__ __forceinline__ double pivot_rsqrt(double d)
{
    if (!f32_range(d)) return 1.0 / sqrt(d);
    const float f = f64_to_f32_trunc(d);
    float y = rsqrtf(f);
    y = y * (1.5f - 0.5f * f * y * y);
    const double yd = f32_to_f64_bits(y);  // y is positive and normal
    const double h = __hiloint2double(__double2hiint(yd) - (1 << 20), __double2loint(yd));  // yd / 2
    const double p = d * yd;
    return fma(h, fma(-p, yd, 1.0), yd);
}

// N = S^-1 for the symmetrised 6 x 6 S by Gauss-Jordan without pivoting, run
// by one whole warp: lane b < 12 holds column b of [S | I] in registers (one
// reciprocal per pivot, the eliminations as shuffles and FMAs).  Returns 1 in
// every lane when a pivot falls below 1e-12 of the largest diagonal entry: a
// body that cannot resist some rigid motion (e.g. blobs on a line through
// the tracking point cannot resist spin about it).  Writes Nm (row-major)
// otherwise.
__device__ int inverse6_warp(const double *__restrict__ S, double *__restrict__ Nm, int lane)
{
    double col[6];
#pragma unroll
    for (int a = 0; a < 6; ++a)
        col[a] = lane < 6 ? 0.5 * (S[a * 6 + lane] + S[lane * 6 + a]) : (lane - 6 == a ? 1.0 : 0.0);
    // the largest |diagonal entry| and the pivot tests on bit patterns
    // (integer compares: non-negative doubles order as their bits), the
    // reciprocal by pivot_rcp: few FP64 instructions on this serial path
    long long bmax = 0;
#pragma unroll
    for (int a = 0; a < 6; ++a)
        bmax = max(bmax, __double_as_longlong(__shfl_sync(0xffffffffu, col[a], a)) &
                             0x7fffffffffffffffLL);
    const long long tb = __double_as_longlong(1e-12 * __longlong_as_double(bmax));
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const double d = __shfl_sync(0xffffffffu, col[c], c);
        const long long db = __double_as_longlong(d);
        if (!(db > tb && db < 0x7ff0000000000000LL)) return 1;  // the same value in every lane
        const double rc = col[c] * pivot_rcp(d);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            if (a == c) continue;
            const double f = __shfl_sync(0xffffffffu, col[a], c);  // A[a][c]
            col[a] -= f * rc;
        }
        col[c] = rc;
    }
    if (lane >= 6 && lane < 12)
#pragma unroll
        for (int a = 0; a < 6; ++a) Nm[a * 6 + lane - 6] = col[a];
    return 0;
}


// Row and column of entry e of a lower triangle enumerated row by row
// (e = i (i + 1) / 2 + j, j <= i).
__device__ __forceinline__ void tri_index(int e, int &i, int &j)
{
    i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while (i > 0 && i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    j = e - i * (i + 1) / 2;
}

// Shared-memory layout of the setup kernel:
//   [L (n*n, only if in smem) | Q (n*6) | QN (n*6) | S (36) | N (36) | dW (n)]
template <bool WALL, bool L_SMEM>
__global__ void __launch_bounds__(kSetupThreads) precond_setup_kernel(
    int64_t nb, const double *__restrict__ r, const double *__restrict__ q,
    const int64_t *__restrict__ start, const int64_t *__restrict__ poff, PairConsts<double> k,
    double scale, double *__restrict__ P, double *__restrict__ scratch, int64_t scratch_stride,
    int *__restrict__ flag, int flag_slot, int schur, const double *__restrict__ shift)
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
        double *dW = Nm + 36;  // diagonal of W = L^-1
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
                    L[(3 * bi + al) * n + 3 * bj + be] =
                        scale * blk[3 * al + be] +
                        (shift && bi == bj && al == be ? shift[b0 + bi] : 0.0);
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
            for (int e = threadIdx.x; e < w * (w + 1) / 2; e += blockDim.x) {
                int i, j;
                tri_index(e, i, j);
                i += c + 1;
                j += c + 1;
                L[i * n + j] -= L[i * n + c] * L[j * n + c];
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

        // 3. W = L^-1 (lower triangular), row by row: row k of W is
        //    (e_k - sum_{j<k} L[k][j] W[j][:]) / L[k][k].  Right-looking: once
        //    row k is complete, subtract its multiples from every later row, so
        //    each step is one parallel sweep.  W[i][c] (i > c) is stored at
        //    L[c][i], the free upper triangle; the diagonal in dW.  Rows are
        //    kept unscaled until the end (W[k][c] = stored * dW[k]).
        for (int i = threadIdx.x; i < n; i += blockDim.x) dW[i] = 1.0 / L[i * n + i];
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int c = e / n, i = e % n;
            if (i > c) L[c * n + i] = 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk + 1 < n; ++kk) {
            const int rows = n - kk - 1, cols = kk + 1;
            const double dk = dW[kk];
            for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
                const int c = e / rows, i = kk + 1 + e % rows;
                const double wkc = c < kk ? L[c * n + kk] * dk : dk;  // W[k][c]
                L[c * n + i] -= L[i * n + kk] * wkc;
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int c = e / n, i = e % n;
            if (i > c) L[c * n + i] *= dW[i];
        }
        __syncthreads();

        // 3b. X = M_p^-1 = W^T W: X[i][j] = sum_{k >= max(i,j)} W[k][i] W[k][j],
        //     written to P_p[:n, :n] (row stride m), both triangles
        for (int e = threadIdx.x; e < n * (n + 1) / 2; e += blockDim.x) {
            int i, j;
            tri_index(e, i, j);  // j <= i
            double acc = dW[i] * (j < i ? L[j * n + i] : dW[i]);
            for (int kk = i + 1; kk < n; ++kk) acc += L[i * n + kk] * L[j * n + kk];
            Pp[(size_t)i * m + j] = acc;
            Pp[(size_t)j * m + i] = acc;
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

        // 6. N = S^-1 on the symmetrised S (warp 0)
        if (threadIdx.x < 32) {
            const int f = inverse6_warp(S, Nm, threadIdx.x);
            if (threadIdx.x == 0 && f) bad = schur;
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
                v = schur ? Pp[(size_t)i * m + j] - acc : Pp[(size_t)i * m + j];
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

// z_p = P_p^-1 [w_p; g_p] for every body.  Work items are (body, row chunk)
// with `chunks` chunks of `rows` rows per body (one chunk when bodies are
// plentiful, several when few bodies would leave SMs idle); one warp per
// output row, lanes across the row.
__global__ void pc_to_f32_kernel(const double *__restrict__ a, int64_t count, float *__restrict__ b)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
         e += (int64_t)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}

// TP: the blocks' type, FP64, or FP32 (an FP32 copy of the explicit blocks
// for the FP32 inner iterations of mixed precision; products and sums in
// FP32 too).
template <typename TP>
__global__ void __launch_bounds__(256) precond_apply_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    const TP *__restrict__ P, const double *__restrict__ w, const double *__restrict__ g,
    double *__restrict__ lam, double *__restrict__ UO, int chunks, int rows, int body_rows)
{
    // body_rows = 6: the indefinite block on [w_p; g_p]; 0: the blob block
    // M_pp^-1 alone on w_p (the resistance problem's preconditioner)
    extern __shared__ double xs_raw[];
    TP *xs = (TP *)xs_raw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t item = blockIdx.x; item < nb * chunks; item += gridDim.x) {
        const int64_t p = item / chunks;
        const int r0 = (int)(item % chunks) * rows;
        const int64_t b0 = start[p];
        const int n = 3 * (int)(start[p + 1] - b0);
        const int m = n + 6, me = n + body_rows;  // stored stride, rows used
        const int r1 = min(me, r0 + rows);
        if (r0 >= me) continue;  // uniform over the CTA
        __syncthreads();
        for (int e = threadIdx.x; e < me; e += blockDim.x)
            xs[e] = TP(e < n ? w[3 * b0 + e] : g[6 * p + (e - n)]);
        __syncthreads();
        const TP *Pp = P + poff[p];
        for (int row = r0 + warp; row < r1; row += nw) {
            const TP *pr = Pp + (size_t)row * m;
            TP acc = TP(0);
            for (int c = lane; c < me; c += 32) acc += pr[c] * xs[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                if (row < n) lam[3 * b0 + row] = double(acc);
                else UO[6 * p + (row - n)] = double(acc);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Split setup for bodies with 3 n_p <= kSplitMaxRows.  The single kernel
// above runs every step of a body on one SM; here only the Cholesky does,
// and the O(n^3) rest is spread over many CTAs:
//   S1 pc_assemble_kernel  M_p's lower triangle written into P_p's n x n block
//                          (warp per blob row and 32 columns);
//   S2 pc_factor_kernel    one CTA per body: Cholesky M_p = L L^T carried out
//                          together with G = L^-1 K_p (the six K columns are
//                          eliminated alongside), then S = G^T G = K^T M^-1 K,
//                          N = S^-1; stores L^T in P_p's upper triangle;
//   S3 pc_trinv_kernel     one warp per column c of W = L^-1 (forward
//                          substitution in registers), with row c of
//                          Q = M^-1 K = W^T G and of Q N, and P_p's border;
//   S4 pc_product_kernel   P_p's n x n block = W^T W - (Q N) Q^T in 32 x 32
//                          tiles through shared memory.
// Per-body scratch (stride kept uniform within a group of bodies):
//   [W (nmax^2, row-major, zero above the diagonal near it) | G (6 nmax) |
//    Q (6 nmax) | QN (6 nmax) | dW (nmax) | N (36)].
constexpr int kSplitMaxRows = 512;
constexpr int kTile = 32;
constexpr int kPanel = 8;  // columns per panel of the shared-memory Cholesky

__device__ __forceinline__ int64_t owner_body(const int64_t *__restrict__ start, int64_t nb,
                                              int64_t b)
{
    int64_t lo = 0, hi = nb;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}

struct SplitScratch {
    double *base;
    int64_t stride;  // doubles per body
    int nmax;
    __device__ double *W(int64_t p) const { return base + p * stride; }
    __device__ double *G(int64_t p) const { return W(p) + (int64_t)nmax * nmax; }
    __device__ double *Q(int64_t p) const { return G(p) + 6 * nmax; }
    __device__ double *QN(int64_t p) const { return Q(p) + 6 * nmax; }
    __device__ double *dW(int64_t p) const { return QN(p) + 6 * nmax; }
    __device__ double *N(int64_t p) const { return dW(p) + nmax; }
};

int64_t split_stride(int nmax) { return (int64_t)nmax * nmax + 19 * (int64_t)nmax + 36; }

// S1: M_p (scaled) into P_p[0:n, 0:n], row stride m = n + 6: the blocks on
// and below the diagonal (bj <= bi), the only ones the factorisations read
// (M_p is symmetric), one warp per blob row and 32 columns (blockIdx.y).
// Launched with small CTAs so that the rows of a few bodies still reach
// every SM: the blocks' dependent FP64 arithmetic is the cost.
template <bool WALL>
__global__ void __launch_bounds__(256) pc_assemble_kernel(
    int64_t nb, const double *__restrict__ r, const int64_t *__restrict__ start,
    const int64_t *__restrict__ poff, PairConsts<double> k, double scale, double *__restrict__ P,
    const double *__restrict__ shift)
{
    const int lane = threadIdx.x & 31;
    const int64_t s0 = start[0], rows = start[nb] - s0;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t it = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); it < rows;
         it += warps) {
        const int64_t b = s0 + it;
        const int64_t p = owner_body(start, nb, b);
        const int64_t b0 = start[p];
        const int np = (int)(start[p + 1] - b0), bi = (int)(b - b0);
        const int m = 3 * np + 6;
        double *Pp = P + poff[p];
        const int bj = 32 * (int)blockIdx.y + lane;
        if (bj <= bi) {
            double blk[9];
            block_f64<WALL>(r + 3 * b, r + 3 * (b0 + bj), k, blk);
#pragma unroll
            for (int al = 0; al < 3; ++al)
#pragma unroll
                for (int be = 0; be < 3; ++be)
                    Pp[(size_t)(3 * bi + al) * m + 3 * bj + be] =
                        scale * blk[3 * al + be] + (shift && bi == bj && al == be ? shift[b] : 0.0);
        }
    }
}

// Entry (row, col) of K_p (rows 3 i + al of blob i are [I, -[d_i]x],
// d_i = r_i - q_p); rb points at the body's first blob.
__device__ __forceinline__ double k_entry(const double *__restrict__ rb, double qx, double qy,
                                          double qz, int row, int col)
{
    const int i = row / 3, al = row % 3;
    if (col < 3) return al == col ? 1.0 : 0.0;
    const double dx = rb[3 * i] - qx, dy = rb[3 * i + 1] - qy, dz = rb[3 * i + 2] - qz;
    // -[d]x = [[0, dz, -dy], [-dz, 0, dx], [dy, -dx, 0]]
    const int e3 = 3 * al + col - 3;
    return e3 == 1 ? dz : e3 == 2 ? -dy : e3 == 3 ? -dz : e3 == 5 ? dx
         : e3 == 6 ? dy : e3 == 7 ? -dx : 0.0;
}

// S2: one CTA per body.  Right-looking Cholesky on the lower triangle with
// the six columns B = K_p appended (so that B ends as G = L^-1 K_p): step c
// scales column c by 1/sqrt(d_c), then subtracts its outer product from the
// trailing triangle and its multiples of row c from the rows of B below,
// one FP64 FMA per entry (FP64 issue is the bound on this chip).  Blocks in
// shared memory take the steps in panels of kPanel columns; blocks in global
// memory use the left-looking order.
template <bool L_SMEM>
__global__ void __launch_bounds__(256) pc_factor_kernel(
    int64_t nb, const double *__restrict__ r, const double *__restrict__ q,
    const int64_t *__restrict__ start, const int64_t *__restrict__ poff, double *__restrict__ P,
    SplitScratch scr, int *__restrict__ flag, int flag_slot, int64_t p_base, int schur)
{
    extern __shared__ double sm[];
    __shared__ int bad, pfail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t p = blockIdx.x; p < nb; p += gridDim.x) {
        const int64_t b0 = start[p];
        const int np = (int)(start[p + 1] - b0);
        const int n = 3 * np, m = n + 6;
        double *Pp = P + poff[p];
        double *L = L_SMEM ? sm : Pp;
        const int ld = L_SMEM ? n : m;
        double *B = L_SMEM ? sm + (size_t)n * n : scr.G(p);
        double *ils = L_SMEM ? B + 6 * n : sm;  // 1 / sqrt(d_c)
        double *S = ils + n;
        double *Nm = S + 36;
        double *col = Nm + 36;  // pivot row (global blocks) / kPanel scaled columns (shared)
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        __syncthreads();
        if (threadIdx.x == 0) bad = 0;
        if (L_SMEM)
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
                const int i = e / n, j = e % n;
                if (j <= i) L[e] = Pp[(size_t)i * m + j];
            }
        // B = K_p: rows of blob i are [I, -[d_i]x]
        for (int e = threadIdx.x; e < 6 * n; e += blockDim.x)
            B[e] = k_entry(r + 3 * b0, qx, qy, qz, e / 6, e % 6);
        int fail = 0;
        if constexpr (L_SMEM) {
        // Blocked order: warp 0 factors a panel of kPanel columns (rows c0..n-1)
        // warp-synchronously, keeping the scaled columns transposed in pT
        // (rows read without bank conflicts); then every warp subtracts the
        // panel's rank-kPanel product from the trailing triangle and from
        // the rows of B below the panel.  The same FMAs as column by column,
        // with two CTA barriers per panel instead of two per column.
        double *pT = col;
        for (int c0 = 0; c0 < n; c0 += kPanel) {
            const int w = n - c0 < kPanel ? n - c0 : kPanel;
            __syncthreads();  // the previous trailing update is complete
            if (warp == 0) {
                int f = 0;
                for (int c = c0; c < c0 + w; ++c) {
                    const double d = L[(size_t)c * ld + c];
                    if (!pivot_ok(d)) {  // the same value in every lane
                        f = 1;
                        break;
                    }
                    const double il = pivot_rsqrt(d);
                    if (lane == 0) ils[c] = il;
                    double *pc = pT + (size_t)(c - c0) * n;
                    for (int i = c + lane; i < n; i += 32) {
                        const double v = L[(size_t)i * ld + c] * il;
                        L[(size_t)i * ld + c] = v;
                        pc[i] = v;
                    }
                    if (lane < 6) B[6 * c + lane] *= il;
                    __syncwarp();
                    // the panel's later columns, and the rows of B inside the panel
                    const int ce = c0 + w - 1;
                    for (int i = c + 1 + lane; i < n; i += 32) {
                        const double lic = pc[i];
                        const int top = i < ce ? i : ce;
                        for (int cc = c + 1; cc <= top; ++cc) L[(size_t)i * ld + cc] -= lic * pc[cc];
                    }
                    for (int e = lane; e < 6 * (ce - c); e += 32) {
                        const int i = c + 1 + e / 6, b = e % 6;
                        B[6 * i + b] -= pc[i] * B[6 * c + b];
                    }
                    __syncwarp();
                }
                if (lane == 0) pfail = f;
            }
            __syncthreads();
            if (pfail) {  // uniform
                fail = 1;
                break;
            }
            const int t0 = c0 + w;
            for (int i = t0 + warp; i < n; i += nw) {
                double li[kPanel];
#pragma unroll
                for (int kk = 0; kk < kPanel; ++kk) li[kk] = kk < w ? pT[(size_t)kk * n + i] : 0.0;
                double *Li = L + (size_t)i * ld;
                for (int j = t0 + lane; j <= i; j += 32) {
                    double acc = Li[j];
#pragma unroll
                    for (int kk = 0; kk < kPanel; ++kk)
                        if (kk < w) acc -= li[kk] * pT[(size_t)kk * n + j];
                    Li[j] = acc;
                }
                if (lane < 6) {
                    double acc = B[6 * i + lane];
#pragma unroll
                    for (int kk = 0; kk < kPanel; ++kk)
                        if (kk < w) acc -= li[kk] * B[6 * (c0 + kk) + lane];
                    B[6 * i + lane] = acc;
                }
            }
        }
        } else {
        // Block in global memory: left-looking (Crout) order.  Column j is
        // L[i][j] = (A[i][j] - L[i][0:j] . L[j][0:j]) / L[j][j], one coalesced
        // dot product per row with the pivot row L[j][0:j] in shared memory
        // (`col`); every entry is written once, so the inner loop only loads
        // and the many independent loads in flight hide the memory latency
        // that the right-looking update's read-modify-writes exposed.  Row j
        // of G = L^-1 K follows from the same pivot row.
        for (int c = 0; c < n; ++c) {
            __syncthreads();  // step c - 1 finished with col
            // the pivot row with its diagonal entry: every warp reads A[c][c]
            // from here, since thread 0 overwrites it in L below
            for (int k = threadIdx.x; k <= c; k += blockDim.x) col[k] = L[(size_t)c * ld + k];
            __syncthreads();
            // pivot d = A[c][c] - |L[c][0:c]|^2, computed by every warp alike
            double acc = 0.0;
            for (int k = lane; k < c; k += 32) acc += col[k] * col[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            const double d = col[c] - acc;
            if (!pivot_ok(d)) {  // the same value in every thread
                fail = 1;
                break;
            }
            const double il = pivot_rsqrt(d);
            if (threadIdx.x == 0) {
                ils[c] = il;
                L[(size_t)c * ld + c] = d * il;  // sqrt(d)
            }
            for (int i = c + 1 + warp; i < n; i += nw) {
                const double *Li = L + (size_t)i * ld;
                double dot = 0.0;
                for (int k = lane; k < c; k += 32) dot += Li[k] * col[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                if (lane == 0) L[(size_t)i * ld + c] = (Li[c] - dot) * il;
            }
            if (warp == nw - 1) {
                // G[c][b] = (K[c][b] - L[c][0:c] . G[0:c][b]) / L[c][c]
#pragma unroll
                for (int b = 0; b < 6; ++b) {
                    double g = 0.0;
                    for (int k = lane; k < c; k += 32) g += col[k] * B[6 * k + b];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                    if (lane == 0) B[6 * c + b] = (B[6 * c + b] - g) * il;
                }
            }
        }
        }
        __syncthreads();
        if (fail) {  // uniform: a pivot was not positive
            if (threadIdx.x == 0) {
                if (flag_slot >= 0) flag[flag_slot] = 2;
                else atomicMin(flag, (int)(p_base + p));
            }
            continue;
        }
        // dW, G to scratch; L^T into P_p's upper triangle (row k holds column k of L)
        double *dW = scr.dW(p), *G = scr.G(p);
        for (int i = threadIdx.x; i < n; i += blockDim.x) dW[i] = ils[i];
        if (L_SMEM)
            for (int e = threadIdx.x; e < 6 * n; e += blockDim.x) G[e] = B[e];
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int kk = e / n, i = e % n;
            if (i > kk) Pp[(size_t)kk * m + i] = L[(size_t)i * ld + kk];
            else if (L_SMEM && i == kk) Pp[(size_t)kk * m + kk] = L[(size_t)kk * ld + kk];
        }
        __syncthreads();
        // S = G^T G (symmetric 6 x 6), one warp per entry
        for (int ab = warp; ab < 36; ab += nw) {
            const int a = ab / 6, bb = ab % 6;
            double acc = 0.0;
            for (int i = lane; i < n; i += 32) acc += B[6 * i + a] * B[6 * i + bb];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) S[ab] = acc;
        }
        __syncthreads();
        // N = S^-1 (warp 0)
        if (warp == 0) {
            const int f = inverse6_warp(S, Nm, lane);
            if (lane == 0 && f) bad = schur;
        }
        __syncthreads();
        if (bad) {
            if (threadIdx.x == 0) {
                if (flag_slot >= 0) flag[flag_slot] = 2;
                else atomicMin(flag, (int)(p_base + p));
            }
            continue;
        }
        double *Ns = scr.N(p);
        if (threadIdx.x < 36) {
            Ns[threadIdx.x] = Nm[threadIdx.x];
            Pp[(size_t)(n + threadIdx.x / 6) * m + n + threadIdx.x % 6] = -Nm[threadIdx.x];
        }
    }
}

// S2 on a cluster of kFacCluster CTAs per body, for problems with fewer
// bodies than SMs (one SM per body would leave most of the chip idle, and
// one SM sustains only about 1.7 FP64 FMA per clock).  Rows are dealt cyclically:
// CTA r holds rows i = r + kFacCluster t of M_p (and of B = K_p).  Panel q
// (columns c0 .. c0 + w - 1, t0 = c0 + w) runs in three stages:
//   (A) warp 0 factors the panel's diagonal block, which every CTA holds in
//       shared memory (the same data and arithmetic in every CTA, so the
//       same pivots and the same failure decision).  Meanwhile the warps of
//       the other SM sub-partitions subtract panel q-1's outer product from
//       the CTA's own rows i >= t0 (columns c0 .. i) and their B rows;
//   (B) the CTA's rows i >= t0 solve for their panel entries, and every CTA
//       solves the panel's B rows: triangular solves against the factored
//       block, one row per 8 lanes (lane k holds entry k);
//   (C) after the one cluster barrier of the panel, every CTA gathers the
//       factored panel of the rows below it, and forms the next panel's
//       diagonal block and B rows itself: their owners' current entries
//       (panels < q applied) minus panel q's product.  The owners write the
//       factored block rows and solved B rows back in place.
// The next block's rows are left out of their owners' trailing updates, so
// no CTA writes an entry that another CTA reads between two barriers: the
// barrier of panel q+1 separates the stage-C reads of panel q from the
// owners' next writes of the same entries.  The outputs are those of
// pc_factor_kernel up to rounding (here each entry takes its products in one
// FMA chain).
constexpr int kFacCluster = 8;

size_t factor_cluster_smem(int nmax, bool srows)
{
    const size_t R = (size_t)(nmax + kFacCluster - 1) / kFacCluster;
    return sizeof(double) * ((srows ? R * nmax : 0) + 6 * R + nmax + 2 * kPanel * kPanel +
                             2 * 6 * kPanel + (size_t)kPanel * nmax + 72);
}

// In-place triangular solve of the 8-lane group that holds y (lane k of the
// group: entry k): y_k <- (y_k - sum_{j<k} x_j D[k][j]) / L_kk, column by
// column (x_j, once final, leaves all later entries in one FMA each); dk[j]
// = D[k][j] (j < k), ilk = 1 / L_kk.  All 32 lanes take part in the shuffles.
__device__ __forceinline__ double panel_solve8(double y, const double (&dk)[kPanel], double ilk,
                                               int k, int w, int lane)
{
#pragma unroll
    for (int j = 0; j < kPanel; ++j) {
        if (j < w) {
            if (k == j) y *= ilk;
            const double xj = __shfl_sync(0xffffffffu, y, (lane & ~7) | j);
            if (k > j && k < w) y -= xj * dk[j];
        }
    }
    return y;
}

// SROWS: the rows of M_p sit in the CTAs' shared memory (3 n_p <= 160);
// otherwise they are factored in place in P_p's lower triangle in global
// memory, each CTA updating its own rows and reading the others' rows
// through L2 (ld.global.cg) after the cluster barriers, which order global
// memory at cluster scope as well.
template <bool SROWS>
__global__ void __cluster_dims__(kFacCluster, 1, 1) __launch_bounds__(256, 2) pc_factor_cluster_kernel(
    int64_t nb, const double *__restrict__ r, const double *__restrict__ q,
    const int64_t *__restrict__ start, const int64_t *__restrict__ poff, double *__restrict__ P,
    SplitScratch scr, int *__restrict__ flag, int flag_slot, int64_t p_base, int schur)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int64_t cid = blockIdx.x / kFacCluster, ncl = gridDim.x / kFacCluster;
    const int nmax = scr.nmax;
    const int R = (nmax + kFacCluster - 1) / kFacCluster;
    extern __shared__ double sm[];
    __shared__ int fail_s, bad;
    double *Lr = sm;                    // R x nmax: own rows of M_p, becoming L (SROWS)
    double *Br = SROWS ? Lr + (size_t)R * nmax : sm;  // R x 6: own rows of K_p, becoming G
    double *ils = Br + 6 * R;           // nmax: 1 / L[c][c] (every CTA keeps all)
    double *Db = ils + nmax;            // 2 x kPanel x kPanel: diagonal blocks (by panel parity)
    double *Bb = Db + 2 * kPanel * kPanel;  // 2 x kPanel x 6: the panels' B rows
    double *Pn = Bb + 2 * 6 * kPanel;   // kPanel x nmax: factored panel, transposed
    double *Sp = Pn + (size_t)kPanel * nmax;  // 36: partial G^T G
    double *Nm = Sp + 36;               // 36
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // The trailing update's warps: 1..3 and 5..7, two on each of the SM
    // sub-partitions 1..3 (warp 0 runs the diagonal chain on sub-partition
    // 0; measured, a share for warp 4 there made the update slower).
    constexpr int kHW = 6;
    const int hw = (warp & 3) ? warp - 1 - (warp >> 2) : -1;
    for (int64_t p = cid; p < nb; p += ncl) {
        const int64_t b0 = start[p];
        const int np = (int)(start[p + 1] - b0);
        const int n = 3 * np, m = n + 6;
        const int nown = n > rank ? (n - 1 - rank) / kFacCluster + 1 : 0;
        double *Pp = P + poff[p];
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        // own row li (row rank + kFacCluster li), any row for reading, and the read
        auto own = [&](int li) -> double * {
            return SROWS ? Lr + (size_t)li * nmax : Pp + (size_t)(rank + kFacCluster * li) * m;
        };
        auto row_of = [&](int row) -> const double * {
            return SROWS ? cluster.map_shared_rank(Lr, row % kFacCluster) +
                               (size_t)(row / kFacCluster) * nmax
                         : Pp + (size_t)row * m;
        };
        auto rd = [](const double *a) -> double { return SROWS ? *a : __ldcg(a); };
        auto brow_of = [&](int row) -> const double * {
            return cluster.map_shared_rank(Br, row % kFacCluster) + 6 * (row / kFacCluster);
        };
        if (SROWS) {
            // own rows' lower-triangle entries, loads issued in batches
            constexpr int kLoad = 4;
            const int tot = nown * n;
            for (int base = 0; base < tot; base += kLoad * (int)blockDim.x) {
                double v[kLoad];
                int dst[kLoad];
#pragma unroll
                for (int u = 0; u < kLoad; ++u) {
                    const int e = base + threadIdx.x + u * (int)blockDim.x;
                    const int li = e / n, j = e - li * n, i = rank + kFacCluster * li;
                    dst[u] = e < tot && j <= i ? li * nmax + j : -1;
                    if (dst[u] >= 0) v[u] = Pp[(size_t)i * m + j];
                }
#pragma unroll
                for (int u = 0; u < kLoad; ++u)
                    if (dst[u] >= 0) Lr[dst[u]] = v[u];
            }
        }
        for (int e = threadIdx.x; e < 6 * nown; e += blockDim.x)
            Br[e] = k_entry(r + 3 * b0, qx, qy, qz, rank + kFacCluster * (e / 6), e % 6);
        cluster.sync();  // every CTA's rows are in place
        // the first diagonal block and its B rows from their owners
        for (int e = threadIdx.x; e < kPanel * kPanel + 6 * kPanel; e += blockDim.x) {
            if (e < kPanel * kPanel) {
                const int a = e / kPanel, b = e % kPanel;
                if (a < n && b <= a) Db[e] = rd(row_of(a) + b);
            } else {
                const int eb = e - kPanel * kPanel, a = eb / 6;
                if (a < n) Bb[eb] = brow_of(a)[eb % 6];
            }
        }
        __syncthreads();
        int fail = 0;
        for (int c0 = 0, par = 0; c0 < n; c0 += kPanel, par ^= 1) {
            const int w = n - c0 < kPanel ? n - c0 : kPanel, t0 = c0 + w;
            double *D = Db + par * kPanel * kPanel, *Bd = Bb + par * 6 * kPanel;
            // own rows below the panel: li >= li0
            const int li0 = t0 > rank ? (t0 - rank + kFacCluster - 1) / kFacCluster : 0;
            const int nr = nown > li0 ? nown - li0 : 0;
            if (warp == 0) {
                // (A) the block's Cholesky on registers: lane l + 8 g holds
                // entries (l, g) and (l, g + 4) (v0, v1), so that a pivot
                // costs two FMAs per lane rather than one per later column;
                // the column loop unrolled, the other lanes' entries by
                // shuffles.  Entries above a row's diagonal may take finite
                // junk and are never read.
                const int l = lane & 7, g = lane >> 3;
                double v0 = l < w && g <= l ? D[l * kPanel + g] : 0.0;
                double v1 = l < w && g + 4 <= l ? D[l * kPanel + g + 4] : 0.0;
                int f = 0;
#pragma unroll
                for (int c = 0; c < kPanel; ++c) {
                    if (c < w && !f) {
                        const int sc = 8 * (c & 3);  // lanes of column c: sc .. sc + 7
                        double &vc = c < 4 ? v0 : v1;
                        const double d = __shfl_sync(0xffffffffu, vc, c + sc);
                        if (!pivot_ok(d)) {
                            f = 1;  // the same value in every lane
                        } else {
                            const double il = pivot_rsqrt(d);
                            if (lane == 0) ils[c0 + c] = il;
                            vc *= g == (c & 3) && l >= c ? il : 1.0;  // lane (c, .): sqrt(d)
                            double lac = __shfl_sync(0xffffffffu, vc, l + sc);  // L[l][c]
                            lac = l > c && l < w ? lac : 0.0;
                            if (c < 4) {
                                const double x0 = __shfl_sync(0xffffffffu, vc, g + sc);  // L[g][c]
                                v0 -= (g > c ? lac : 0.0) * x0;
                            }
                            const double x1 = __shfl_sync(0xffffffffu, vc, g + 4 + sc);  // L[g+4][c]
                            v1 -= (g + 4 > c ? lac : 0.0) * x1;
                        }
                    }
                }
                if (l < w) {
                    if (g <= l) D[l * kPanel + g] = v0;
                    if (g + 4 <= l) D[l * kPanel + g + 4] = v1;
                }
                if (lane == 0) fail_s = f;
            } else if (hw >= 0 && c0 > 0) {
                // (A) the previous panel's product out of own rows i >= t0
                // (columns c0 .. i) and out of their B rows, in items of 32
                // entries (one per lane, one FMA chain each) dealt to the
                // warps in turn: row q's ceil((i - c0 + 1) / 32) items, then
                // the B rows' ceil(6 nr / 32)
                const int cp = c0 - kPanel;  // the previous panel is full
                const double *Bp = Bb + (par ^ 1) * 6 * kPanel;
                int item = 0;
                for (int qq = 0; qq < nr; ++qq) {
                    const int li = li0 + qq, i = rank + kFacCluster * li;
                    const int nit = (i - c0 + 32) >> 5, it0 = item;
                    item += nit;
                    int it = it0 + ((hw - it0) % kHW + kHW) % kHW;  // this warp's first item here
                    if (it >= item) continue;
                    double *Li = own(li);
                    double lk[kPanel];
#pragma unroll
                    for (int k = 0; k < kPanel; ++k) lk[k] = Li[cp + k];
                    for (; it < item; it += kHW) {
                        const int j = c0 + 32 * (it - it0) + lane;
                        if (j <= i) {
                            double a0 = Li[j];
#pragma unroll
                            for (int k = 0; k < kPanel; ++k) a0 -= lk[k] * Pn[(size_t)k * nmax + j];
                            Li[j] = a0;
                        }
                    }
                }
                const int itb = item + ((hw - item) % kHW + kHW) % kHW;
                for (int e = 32 * (itb - item) + lane; e < 6 * nr; e += 32 * kHW) {
                    const int li = li0 + e / 6, x = e % 6;
                    const double *Li = own(li) + cp;
                    double a0 = Br[6 * li + x];
#pragma unroll
                    for (int k = 0; k < kPanel; ++k) a0 -= Li[k] * Bp[6 * k + x];
                    Br[6 * li + x] = a0;
                }
            }
            __syncthreads();
            if (fail_s) {  // uniform over the cluster
                cluster.sync();  // no CTA still reads another's rows
                fail = 1;
                break;
            }
            // (B) the panel's B rows (groups 0..5, column x = group) and own
            // rows i >= t0 (groups 6..), solved against the factored block
            {
                const int k = lane & 7, ng = nr + 6;
                double dk[kPanel];
#pragma unroll
                for (int j = 0; j < kPanel; ++j) dk[j] = j < k && k < w ? D[k * kPanel + j] : 0.0;
                const double ilk = k < w ? ils[c0 + k] : 0.0;
                for (int g0 = 4 * warp; g0 < ng; g0 += 4 * nw) {  // uniform over the warp
                    const int g = g0 + (lane >> 3);
                    double *dst = nullptr;
                    double y = 0.0;
                    if (g < ng && k < w) {
                        dst = g < 6 ? Bd + 6 * k + g : own(li0 + g - 6) + c0 + k;
                        y = *dst;
                    }
                    y = panel_solve8(y, dk, ilk, k, w, lane);
                    if (dst) *dst = y;
                }
            }
            cluster.sync();  // every CTA's panel entries are final
            // (C) warps 0..4: the factored panel of rows t0..n-1 from their
            // owners into Pn (remote loads issued in batches of kGather per
            // thread before any store, so that their latencies overlap)
            const int w2 = n - t0 < kPanel ? n - t0 : kPanel;  // the next panel's width
            if (warp < 5) {
                constexpr int kGather = 8;
                const int total = (n - t0) * w, nt = 5 * 32;
                for (int base = 0; base < total; base += kGather * nt) {
                    double v[kGather];
                    int dst[kGather];
#pragma unroll
                    for (int u = 0; u < kGather; ++u) {
                        const int e = base + threadIdx.x + u * nt;
                        dst[u] = -1;
                        if (e < total) {
                            const int j = t0 + e / w, k = e % w;
                            v[u] = rd(row_of(j) + c0 + k);
                            dst[u] = k * nmax + j;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kGather; ++u)
                        if (dst[u] >= 0) Pn[dst[u]] = v[u];
                }
            } else if (w2 > 0) {
                // warps 5..7: the next diagonal block (entry (a, b), b <= a,
                // 36 of them) and its B rows (entry (a, x), 48): the owners'
                // entries minus this panel's product, which is full here
                double *Dn = Db + (par ^ 1) * kPanel * kPanel, *Bn = Bb + (par ^ 1) * 6 * kPanel;
                const int e = threadIdx.x - 5 * 32;
                constexpr int kTri = kPanel * (kPanel + 1) / 2;
                if (e < kTri) {
                    int a = 0;
                    while ((a + 1) * (a + 2) / 2 <= e) ++a;
                    const int b = e - a * (a + 1) / 2;
                    if (a < w2) {
                        const double *ra = row_of(t0 + a), *rb = row_of(t0 + b);
                        double la[kPanel], lb[kPanel];
#pragma unroll
                        for (int k = 0; k < kPanel; ++k) {
                            la[k] = rd(ra + c0 + k);
                            lb[k] = rd(rb + c0 + k);
                        }
                        double a0 = rd(ra + t0 + b);
#pragma unroll
                        for (int k = 0; k < kPanel; ++k) a0 -= la[k] * lb[k];
                        Dn[a * kPanel + b] = a0;
                    }
                } else if (e < kTri + 6 * kPanel) {
                    const int a = (e - kTri) / 6, x = (e - kTri) % 6;
                    if (a < w2) {
                        const double *ra = row_of(t0 + a);
                        double la[kPanel];
#pragma unroll
                        for (int k = 0; k < kPanel; ++k) la[k] = rd(ra + c0 + k);
                        double a0 = brow_of(t0 + a)[x];
#pragma unroll
                        for (int k = 0; k < kPanel; ++k) a0 -= la[k] * Bd[6 * k + x];
                        Bn[6 * a + x] = a0;
                    }
                }
            }
            // the owners of the block's rows store its factored rows and B rows
            for (int e = threadIdx.x; e < kPanel * kPanel + 6 * kPanel; e += blockDim.x) {
                if (e < kPanel * kPanel) {
                    const int a = e / kPanel, b = e % kPanel, row = c0 + a;
                    if (a < w && b <= a && row % kFacCluster == rank)
                        own(row / kFacCluster)[c0 + b] = D[e];
                } else {
                    const int eb = e - kPanel * kPanel, row = c0 + eb / 6;
                    if (eb / 6 < w && row % kFacCluster == rank)
                        Br[6 * (row / kFacCluster) + eb % 6] = Bd[eb];
                }
            }
            __syncthreads();
        }
        if (fail) {
            if (rank == 0 && threadIdx.x == 0) {
                if (flag_slot >= 0) flag[flag_slot] = 2;
                else atomicMin(flag, (int)(p_base + p));
            }
            continue;
        }
        __syncthreads();
        // own rows: L^T into P_p's upper triangle (row k holds column k of L),
        // 1 / L[i][i] and G to the scratch
        double *dW = scr.dW(p), *G = scr.G(p);
        for (int e = threadIdx.x; e < nown * n; e += blockDim.x) {
            const int li = e / n, k = e % n, i = rank + kFacCluster * li;
            if (k <= i) Pp[(size_t)k * m + i] = own(li)[k];
        }
        for (int li = threadIdx.x; li < nown; li += blockDim.x) {
            const int i = rank + kFacCluster * li;
            dW[i] = ils[i];
        }
        for (int e = threadIdx.x; e < 6 * nown; e += blockDim.x) {
            const int li = e / 6, i = rank + kFacCluster * li;
            G[6 * i + e % 6] = Br[e];
        }
        // partial S = G^T G over own rows, one warp per entry
        for (int ab = warp; ab < 36; ab += nw) {
            const int a = ab / 6, bb = ab % 6;
            double acc = 0.0;
            for (int li = lane; li < nown; li += 32) acc += Br[6 * li + a] * Br[6 * li + bb];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) Sp[ab] = acc;
        }
        cluster.sync();  // every CTA's partial S is written
        if (rank == 0) {
            // S summed over the cluster in rank order; N = S^-1
            if (threadIdx.x < 36) {
                double acc = 0.0;
                for (int rr = 0; rr < kFacCluster; ++rr)
                    acc += cluster.map_shared_rank(Sp, rr)[threadIdx.x];
                Db[threadIdx.x] = acc;  // the 36 entries of S (the blocks are free now)
            }
            __syncthreads();
            if (warp == 0) {
                const int f = inverse6_warp(Db, Nm, lane);
                if (lane == 0) bad = f ? schur : 0;
            }
            __syncthreads();
            if (bad) {
                if (threadIdx.x == 0) {
                    if (flag_slot >= 0) flag[flag_slot] = 2;
                    else atomicMin(flag, (int)(p_base + p));
                }
            } else if (threadIdx.x < 36) {
                scr.N(p)[threadIdx.x] = Nm[threadIdx.x];
                Pp[(size_t)(n + threadIdx.x / 6) * m + n + threadIdx.x % 6] = -Nm[threadIdx.x];
            }
        }
        cluster.sync();  // rank 0 has read every partial S
    }
}

// S3: warp per column c of W = L^-1.  Lane l holds rows 32 t + l of the
// column (t < R).  Step k: W[k][c] = (current value of row k) / L[k][k],
// then rows i > k lose L[i][k] W[k][c].  L[i][k] is read from P_p's upper
// triangle (contiguous in i).  Along the way the warp forms
// Q[c][:] = sum_k W[k][c] G[k][:] and QN[c][:] = Q[c][:] N, and writes P_p's
// border entries -QN[c][b] (column n + b of row c and its transpose).
template <int R>
__global__ void __launch_bounds__(256) pc_trinv_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    double *__restrict__ P, SplitScratch scr, int col_groups)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t item = blockIdx.x; item < nb * col_groups; item += gridDim.x) {
        const int64_t p = item / col_groups;
        const int c = (int)(item % col_groups) * nw + warp;
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        if (c >= n) continue;  // warp-uniform
        const double *Lt = P + poff[p];
        double *W = scr.W(p);
        const double *G = scr.G(p), *dW = scr.dW(p), *Nm = scr.N(p);
        const int ldw = scr.nmax;
        double w[R];
#pragma unroll
        for (int t = 0; t < R; ++t) w[t] = (32 * t + lane == c) ? 1.0 : 0.0;
        // zero the rows of column c that the tiled product reads above the diagonal
        for (int kk = (c & ~(kTile - 1)) + lane; kk < c; kk += 32) W[(size_t)kk * ldw + c] = 0.0;
        double qa = 0.0;  // lane b < 6: Q[c][b]
#pragma unroll
        for (int t = 0; t < R; ++t) {
            if (32 * t + 31 < c) continue;
            if (32 * t >= n) break;
            for (int l = 0; l < 32; ++l) {
                const int k = 32 * t + l;
                if (k < c) continue;
                if (k >= n) break;
                const double wk = __shfl_sync(0xffffffffu, w[t], l) * dW[k];
                if (lane == l) W[(size_t)k * ldw + c] = wk;
                if (lane < 6) qa += wk * G[6 * k + lane];
                const double *lk = Lt + (size_t)k * m;
#pragma unroll
                for (int t2 = t; t2 < R; ++t2) {
                    const int i = 32 * t2 + lane;
                    if (i > k && i < n) w[t2] -= lk[i] * wk;
                }
            }
        }
        // QN[c][b] = sum_a Q[c][a] N[a][b]
        double qn = 0.0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            const double qv = __shfl_sync(0xffffffffu, qa, a);
            if (lane < 6) qn += qv * Nm[a * 6 + lane];
        }
        if (lane < 6) {
            scr.Q(p)[6 * c + lane] = qa;
            scr.QN(p)[6 * c + lane] = qn;
            P[poff[p] + (size_t)c * m + n + lane] = -qn;
            P[poff[p] + (size_t)(n + lane) * m + c] = -qn;
        }
    }
}

// ---------------------------------------------------------------------------
// S3 and S4 in double-float for blocks of up to 4 kTile rows.  On this chip an
// FP64 warp instruction issues about once per 19 SM cycles, so the
// substitution chains of S3 (a few FP64 instructions per step, one step per
// row) and the 32 x 32 x 32 tiles of S4 are bound by FP64 issue, not by
// their arithmetic.  Double-float arithmetic (df32.cuh: about 46 bits, each
// operation a few FP32 instructions) carries W = L^-1, Q = W^T G, Q N and
// W^T W - (Q N) Q^T on the FP32 pipes instead; the Cholesky factor, G and N
// come from the FP64 factorisation, and the stored inverse is FP64.  Its
// entries then carry a relative error of about 1e-14 (a few double-float
// roundings per step over n steps) instead of FP64 rounding: the
// preconditioner changes the iteration count, not the solution, which the
// flexible GMRES takes from true residuals.
//
// S2' converts, in place, the FP64 inputs of S3 to double-float pairs packed
// in the same 8 bytes: the rows of L^T in P_p's upper triangle, and dW, G and
// N in the scratch.
__device__ __forceinline__ double df_pack(dfl v)
{
    return __hiloint2double(__float_as_int(v.hi), __float_as_int(v.lo));
}

__device__ __forceinline__ dfl df_unpack(double d)
{
    return dfl(__int_as_float(__double2hiint(d)), __int_as_float(__double2loint(d)));
}

__device__ __forceinline__ dfl df_of(double d)
{
    const float h = (float)d;
    return dfl(h, (float)(d - (double)h));
}

__global__ void __launch_bounds__(256) pc_to_df_kernel(int64_t nb,
                                                       const int64_t *__restrict__ start,
                                                       const int64_t *__restrict__ poff,
                                                       double *__restrict__ P, SplitScratch scr)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t rows = nb * scr.nmax;
    for (int64_t it = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); it < rows;
         it += warps) {
        const int64_t p = it / scr.nmax;
        const int k = (int)(it % scr.nmax);
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        if (k >= n) continue;
        double *Lk = P + poff[p] + (size_t)k * m;
        for (int i = k + 1 + lane; i < n; i += 32) Lk[i] = df_pack(df_of(Lk[i]));
        if (lane == 0) scr.dW(p)[k] = df_pack(df_of(scr.dW(p)[k]));
        if (lane < 6) scr.G(p)[6 * k + lane] = df_pack(df_of(scr.G(p)[6 * k + lane]));
        if (k == 0)
            for (int e = lane; e < 36; e += 32) scr.N(p)[e] = df_pack(df_of(scr.N(p)[e]));
    }
}

__device__ __forceinline__ void cp_async8(double *smem, const double *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Offset of row k of the staged triangle (rows cmin ..), n rows in all
__device__ __forceinline__ int tri_row_off(int k, int cmin, int n)
{
    return (k - cmin) * (2 * (n - 1) - (cmin + k - 1)) / 2;
}

// S3 in double-float: warp per column c of W = L^-1, rows 32 t + lane in
// registers, as pc_trinv_kernel; W, Q and Q N go to the scratch as packed
// double-float, the border entries -Q N of P_p in FP64.  1 / L_kk travels
// through the chain by shuffles from registers.  L^T and G are read from
// L2: this form serves many bodies, whose CTAs stay small; few bodies take
// pc_trinv_df_pair_kernel.
__global__ void __launch_bounds__(256) pc_trinv_df_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    double *__restrict__ P, SplitScratch scr, int col_groups)
{
    constexpr int R = 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t item = blockIdx.x; item < nb * col_groups; item += gridDim.x) {
        const int64_t p = item / col_groups;
        const int cmin = (int)(item % col_groups) * nw;
        const int c = cmin + warp;
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        // row k of L^T at Lk + (k - cmin) * ldl, row k of G at Gk + 6 (k - cmin)
        const double *Lk = P + poff[p] + (size_t)cmin * m, *Gk = scr.G(p) + 6 * cmin;
        const int ldl = m;
        if (c >= n) continue;  // warp-uniform
        double *W = scr.W(p);
        const double *dW = scr.dW(p), *Nm = scr.N(p);
        const int ldw = scr.nmax;
        dfl w[R];
#pragma unroll
        for (int t = 0; t < R; ++t) w[t] = dfl((32 * t + lane == c) ? 1.f : 0.f, 0.f);
        // zero the rows of column c that the tiled product reads above the diagonal
        for (int kk = (c & ~(kTile - 1)) + lane; kk < c; kk += 32) W[(size_t)kk * ldw + c] = 0.0;
        dfl qa;  // lane b < 6: Q[c][b]
        // 1 / L_kk of rows 32 t + lane in registers (passed by shuffles in the chain)
        dfl dwr[R];
#pragma unroll
        for (int t = 0; t < R; ++t) dwr[t] = 32 * t + lane < n ? df_unpack(dW[32 * t + lane]) : dfl();
        {
#pragma unroll
            for (int t = 0; t < R; ++t) {
                if (32 * t + 31 < c) continue;
                if (32 * t >= n) break;
                for (int l = 0; l < 32; ++l) {
                    const int k = 32 * t + l;
                    if (k < c) continue;
                    if (k >= n) break;
                    const dfl wl(__shfl_sync(0xffffffffu, w[t].hi, l), __shfl_sync(0xffffffffu, w[t].lo, l));
                    const dfl dk(__shfl_sync(0xffffffffu, dwr[t].hi, l), __shfl_sync(0xffffffffu, dwr[t].lo, l));
                    const dfl wk = wl * dk;
                    if (lane == l) W[(size_t)k * ldw + c] = df_pack(wk);
                    if (lane < 6) qa += wk * df_unpack(Gk[6 * (k - cmin) + lane]);
                    const double *lk = Lk + (size_t)(k - cmin) * ldl;  // row k of L^T
#pragma unroll
                    for (int t2 = t; t2 < R; ++t2) {
                        const int i = 32 * t2 + lane;
                        if (i > k && i < n) w[t2] = w[t2] - df_unpack(lk[i]) * wk;
                    }
                }
            }
        }
        // QN[c][b] = sum_a Q[c][a] N[a][b]
        dfl qn;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            const dfl qv(__shfl_sync(0xffffffffu, qa.hi, a), __shfl_sync(0xffffffffu, qa.lo, a));
            if (lane < 6) qn += qv * df_unpack(Nm[a * 6 + lane]);
        }
        if (lane < 6) {
            scr.Q(p)[6 * c + lane] = df_pack(qa);
            scr.QN(p)[6 * c + lane] = df_pack(qn);
            const double v = -to_double(qn);
            P[poff[p] + (size_t)c * m + n + lane] = v;
            P[poff[p] + (size_t)(n + lane) * m + c] = v;
        }
    }
}

// One 32-row tile t of a column's chain (the steps of pc_trinv_df_kernel):
// lane l holds row 32 t + l in wt; the step of row k leaves W[k][c] in lane
// k - 32 t of wst and updates only the tile's own rows.
__device__ __forceinline__ void trinv_tile_chain(int t, int c, int n, int cmin,
                                                 const double *__restrict__ sLt, dfl &wt, dfl dwrt,
                                                 dfl &wst, int lane)
{
    const int i = 32 * t + lane;
    for (int l = 0; l < 32; ++l) {
        const int k = 32 * t + l;
        if (k < c) continue;
        if (k >= n) break;
        const dfl lik = i > k && i < n ? df_unpack(sLt[tri_row_off(k, cmin, n) - (k + 1) + i]) : dfl();
        const dfl wl(__shfl_sync(0xffffffffu, wt.hi, l), __shfl_sync(0xffffffffu, wt.lo, l));
        const dfl dk(__shfl_sync(0xffffffffu, dwrt.hi, l), __shfl_sync(0xffffffffu, dwrt.lo, l));
        const dfl wk = wl * dk;
        wst = lane == l ? wk : wst;
        const dfl wn = wt - lik * wk;
        wt = i > k && i < n ? wn : wt;
    }
}

// S3 in double-float for few bodies (rows n <= 128): four columns per CTA,
// a pair of warps per column.  Warp A holds the column's rows 0..63 (tiles
// 0, 1), warp B rows 64..127 (tiles 2, 3).  The pace is set by a warp's
// instruction count (about 5 cycles each: every step is a dependent chain),
// so the pair splits the column's work in three phases between barriers:
//   1. A runs tile 0's chain and leaves its W entries in shared memory;
//   2. A subtracts tile 0's product from tile 1, runs tile 1 and leaves its
//      entries and Q's sums over tiles 0, 1; meanwhile B subtracts tile 0's
//      product from its rows;
//   3. B subtracts tile 1's product, runs tiles 2 and 3 and carries Q on
//      from A's sums.
// Every entry takes the same operations in the same order as in one warp
// (pc_trinv_df_kernel).  The CTA first copies the rows of L^T its columns
// need (from its first column on; row k holds entries k+1 .. n-1, rows back
// to back, all copies in flight at once by cp.async) and their rows of G
// into shared memory, so that no step of a chain waits on L2.
__global__ void __launch_bounds__(256) pc_trinv_df_pair_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    double *__restrict__ P, SplitScratch scr, int col_groups)
{
    constexpr int kCols = 4;
    extern __shared__ double sLt[];  // L^T rows cmin .. n-1 (packed triangle), G rows, exchange
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int q = warp >> 1, role = warp & 1;
    const int nmax = scr.nmax;
    dfl *xw = (dfl *)(sLt + (size_t)nmax * (nmax - 1) / 2 + 6 * (size_t)nmax);  // [kCols][2][32]
    dfl *xq = xw + kCols * 2 * 32;                                               // [kCols][6]
    for (int64_t item = blockIdx.x; item < nb * col_groups; item += gridDim.x) {
        const int64_t p = item / col_groups;
        const int cmin = (int)(item % col_groups) * kCols;
        const int c = cmin + q;
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        double *sG = sLt + (cmin < n ? tri_row_off(n, cmin, n) : 0);
        __syncthreads();  // the previous item is finished with the shared arrays
        if (cmin < n) {
            // asynchronous copies, all in flight at once: a warp per row
            const double *Lg = P + poff[p];
            for (int k = cmin + warp; k < n; k += nw) {
                double *dst = sLt + tri_row_off(k, cmin, n) - (k + 1);
                for (int i = k + 1 + lane; i < n; i += 32) cp_async8(dst + i, Lg + (size_t)k * m + i);
            }
            for (int e = threadIdx.x; e < 6 * (n - cmin); e += blockDim.x)
                cp_async8(sG + e, scr.G(p) + 6 * cmin + e);
            cp_async_wait_all();
        }
        __syncthreads();
        const bool active = c < n;  // the same in both warps of the pair
        double *W = scr.W(p);
        const double *dW = scr.dW(p), *Nm = scr.N(p);
        const int ldw = scr.nmax;
        // this warp's tiles 2 role + tt: rows 64 role + 32 tt + lane
        dfl w[2], ws[2], dwr[2];
#pragma unroll
        for (int tt = 0; tt < 2; ++tt) {
            const int i = 64 * role + 32 * tt + lane;
            w[tt] = dfl(i == c ? 1.f : 0.f, 0.f);
            ws[tt] = dfl();
            dwr[tt] = i < n ? df_unpack(dW[i]) : dfl();
        }
        dfl qa;  // lane b < 6: Q[c][b]
        // whether tile t holds steps of column c
        auto has = [&](int t) { return 32 * t + 31 >= c && 32 * t < n; };
        // (1) A: tile 0
        if (active && role == 0) {
            // zero the rows of column c that the tiled product reads above the diagonal
            for (int kk = (c & ~(kTile - 1)) + lane; kk < c; kk += 32) W[(size_t)kk * ldw + c] = 0.0;
            if (has(0)) {
                trinv_tile_chain(0, c, n, cmin, sLt, w[0], dwr[0], ws[0], lane);
                if (lane >= c && lane < n) W[(size_t)lane * ldw + c] = df_pack(ws[0]);
                xw[(q * 2) * 32 + lane] = ws[0];
            }
        }
        __syncthreads();
        if (active && role == 0) {
            // (2) A: tile 0's product out of tile 1 and its share of Q, then tile 1
            if (has(0))
                for (int l = 0; l < 32; ++l) {
                    const int k = l;
                    if (k < c) continue;
                    if (k >= n) break;
                    const dfl wk(__shfl_sync(0xffffffffu, ws[0].hi, l), __shfl_sync(0xffffffffu, ws[0].lo, l));
                    if (lane < 6) qa += wk * df_unpack(sG[6 * (k - cmin) + lane]);
                    const int i1 = 32 + lane;
                    if (i1 < n) w[1] = w[1] - df_unpack(sLt[tri_row_off(k, cmin, n) - (k + 1) + i1]) * wk;
                }
            if (has(1)) {
                trinv_tile_chain(1, c, n, cmin, sLt, w[1], dwr[1], ws[1], lane);
                const int i = 32 + lane;
                if (i >= c && i < n) W[(size_t)i * ldw + c] = df_pack(ws[1]);
                xw[(q * 2 + 1) * 32 + lane] = ws[1];
                for (int l = 0; l < 32; ++l) {
                    const int k = 32 + l;
                    if (k < c) continue;
                    if (k >= n) break;
                    const dfl wk(__shfl_sync(0xffffffffu, ws[1].hi, l), __shfl_sync(0xffffffffu, ws[1].lo, l));
                    if (lane < 6) qa += wk * df_unpack(sG[6 * (k - cmin) + lane]);
                }
            }
            if (lane < 6) xq[q * 6 + lane] = qa;
        } else if (active && role == 1 && has(0)) {
            // (2) B: tile 0's product out of rows 64 .. n-1
            for (int l = 0; l < 32; ++l) {
                const int k = l;
                if (k < c) continue;
                if (k >= n) break;
                const dfl wk = xw[(q * 2) * 32 + l];
                const double *lk = sLt + tri_row_off(k, cmin, n) - (k + 1);
#pragma unroll
                for (int tt = 0; tt < 2; ++tt) {
                    const int i2 = 64 + 32 * tt + lane;
                    if (i2 < n) w[tt] = w[tt] - df_unpack(lk[i2]) * wk;
                }
            }
        }
        __syncthreads();
        if (active && role == 1) {
            // (3) B: tile 1's product out of its rows, then tiles 2 and 3
            qa = lane < 6 ? xq[q * 6 + lane] : dfl();
            if (has(1))
                for (int l = 0; l < 32; ++l) {
                    const int k = 32 + l;
                    if (k < c) continue;
                    if (k >= n) break;
                    const dfl wk = xw[(q * 2 + 1) * 32 + l];
                    const double *lk = sLt + tri_row_off(k, cmin, n) - (k + 1);
#pragma unroll
                    for (int tt = 0; tt < 2; ++tt) {
                        const int i2 = 64 + 32 * tt + lane;
                        if (i2 < n) w[tt] = w[tt] - df_unpack(lk[i2]) * wk;
                    }
                }
#pragma unroll
            for (int tt = 0; tt < 2; ++tt) {
                const int t = 2 + tt;
                if (!has(t)) continue;
                trinv_tile_chain(t, c, n, cmin, sLt, w[tt], dwr[tt], ws[tt], lane);
                const int i = 32 * t + lane;
                if (i >= c && i < n) W[(size_t)i * ldw + c] = df_pack(ws[tt]);
                for (int l = 0; l < 32; ++l) {
                    const int k = 32 * t + l;
                    if (k < c) continue;
                    if (k >= n) break;
                    const dfl wk(__shfl_sync(0xffffffffu, ws[tt].hi, l), __shfl_sync(0xffffffffu, ws[tt].lo, l));
                    if (lane < 6) qa += wk * df_unpack(sG[6 * (k - cmin) + lane]);
                    if (tt == 0) {
                        const int i1 = 96 + lane;
                        if (i1 < n) w[1] = w[1] - df_unpack(sLt[tri_row_off(k, cmin, n) - (k + 1) + i1]) * wk;
                    }
                }
            }
            // QN[c][b] = sum_a Q[c][a] N[a][b]
            dfl qn;
#pragma unroll
            for (int a = 0; a < 6; ++a) {
                const dfl qv(__shfl_sync(0xffffffffu, qa.hi, a), __shfl_sync(0xffffffffu, qa.lo, a));
                if (lane < 6) qn += qv * df_unpack(Nm[a * 6 + lane]);
            }
            if (lane < 6) {
                scr.Q(p)[6 * c + lane] = df_pack(qa);
                scr.QN(p)[6 * c + lane] = df_pack(qn);
                const double v = -to_double(qn);
                P[poff[p] + (size_t)c * m + n + lane] = v;
                P[poff[p] + (size_t)(n + lane) * m + c] = v;
            }
        }
    }
}

// S4 in double-float: P_p's n x n block = W^T W - (Q N) Q^T in TILE x TILE
// tiles (as pc_product_kernel; 16 x 16 when there are few bodies, so that the
// tiles reach more SMs), the tiles of W staged in shared memory as
// double-float, the result stored in FP64.  256 threads: thread (ty, tx)
// forms rows ty + (256 / TILE) rr of the tile's column tx.
template <int TILE>
__global__ void __launch_bounds__(256) pc_product_df_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    double *__restrict__ P, SplitScratch scr, int tiles_per_body, int schur)
{
    constexpr int kRows = 256 / TILE, kRR = TILE / kRows;
    __shared__ dfl Wi[TILE][TILE + 1], Wj[TILE][TILE + 1];
    const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
    for (int64_t item = blockIdx.x; item < nb * tiles_per_body; item += gridDim.x) {
        const int64_t p = item / tiles_per_body;
        int I, J;
        tri_index((int)(item % tiles_per_body), I, J);
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        const int i0 = I * TILE, j0 = J * TILE;
        if (i0 >= n) continue;  // CTA-uniform
        const double *W = scr.W(p);
        const int ldw = scr.nmax;
        dfl acc[kRR];
        for (int k0 = i0; k0 < n; k0 += TILE) {
            __syncthreads();
            for (int e = threadIdx.x; e < TILE * TILE; e += blockDim.x) {
                const int kk = e / TILE, cc = e % TILE;
                const int k = k0 + kk;
                Wi[kk][cc] = (k < n && i0 + cc < n) ? df_unpack(W[(size_t)k * ldw + i0 + cc]) : dfl();
                Wj[kk][cc] = (k < n && j0 + cc < n) ? df_unpack(W[(size_t)k * ldw + j0 + cc]) : dfl();
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < TILE; ++kk) {
                const dfl wj = Wj[kk][tx];
#pragma unroll
                for (int rr = 0; rr < kRR; ++rr) acc[rr] += Wi[kk][ty + kRows * rr] * wj;
            }
        }
        const double *Qs = scr.Q(p), *QN = scr.QN(p);
        double *Pp = P + poff[p];
        const int j = j0 + tx;
#pragma unroll
        for (int rr = 0; rr < kRR; ++rr) {
            const int i = i0 + ty + kRows * rr;
            if (i >= n || j >= n || (I == J && j > i)) continue;
            dfl v = acc[rr];
            if (schur)
#pragma unroll
                for (int bb = 0; bb < 6; ++bb)
                    v = v - df_unpack(QN[6 * i + bb]) * df_unpack(Qs[6 * j + bb]);
            const double vd = to_double(v);
            Pp[(size_t)i * m + j] = vd;
            Pp[(size_t)j * m + i] = vd;
        }
    }
}

// S3 for larger blocks (3 n_p up to kSplitMaxRowsSmem): the same
// substitution with the warp's column in shared memory instead of registers
// (n doubles per warp); __syncwarp orders each step's update before the
// next step's read of the new pivot row.
constexpr int kSplitMaxRowsSmem = 2048;
constexpr int kTrinvSmemWarps = 8;

__global__ void __launch_bounds__(32 * kTrinvSmemWarps) pc_trinv_smem_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    double *__restrict__ P, SplitScratch scr, int col_groups)
{
    extern __shared__ double colbuf[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double *w = colbuf + (size_t)warp * scr.nmax;
    for (int64_t item = blockIdx.x; item < nb * col_groups; item += gridDim.x) {
        const int64_t p = item / col_groups;
        const int c = (int)(item % col_groups) * nw + warp;
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        if (c >= n) continue;  // warp-uniform
        const double *Lt = P + poff[p];
        double *W = scr.W(p);
        const double *G = scr.G(p), *dW = scr.dW(p), *Nm = scr.N(p);
        const int ldw = scr.nmax;
        for (int i = lane; i < n; i += 32) w[i] = i == c ? 1.0 : 0.0;
        for (int kk = (c & ~(kTile - 1)) + lane; kk < c; kk += 32) W[(size_t)kk * ldw + c] = 0.0;
        __syncwarp();
        double qa = 0.0;  // lane b < 6: Q[c][b]
        for (int k = c; k < n; ++k) {
            const double wk = w[k] * dW[k];
            if (lane == 0) W[(size_t)k * ldw + c] = wk;
            if (lane < 6) qa += wk * G[6 * k + lane];
            const double *lk = Lt + (size_t)k * m;
            for (int i = k + 1 + lane; i < n; i += 32) w[i] -= lk[i] * wk;
            __syncwarp();
        }
        double qn = 0.0;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            const double qv = __shfl_sync(0xffffffffu, qa, a);
            if (lane < 6) qn += qv * Nm[a * 6 + lane];
        }
        if (lane < 6) {
            scr.Q(p)[6 * c + lane] = qa;
            scr.QN(p)[6 * c + lane] = qn;
            P[poff[p] + (size_t)c * m + n + lane] = -qn;
            P[poff[p] + (size_t)(n + lane) * m + c] = -qn;
        }
        __syncwarp();  // the next column reuses w
    }
}

// S4: P_p[i][j] = sum_k W[k][i] W[k][j] - sum_b QN[i][b] Q[j][b] on the
// lower 32 x 32 tiles (I >= J) of the n x n block, mirrored to the upper.
__global__ void __launch_bounds__(256) pc_product_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    double *__restrict__ P, SplitScratch scr, int tiles_per_body, int schur)
{
    __shared__ double Wi[kTile][kTile + 1], Wj[kTile][kTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of threads
    for (int64_t item = blockIdx.x; item < nb * tiles_per_body; item += gridDim.x) {
        const int64_t p = item / tiles_per_body;
        int I, J;
        tri_index((int)(item % tiles_per_body), I, J);
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        const int i0 = I * kTile, j0 = J * kTile;
        if (i0 >= n) continue;  // CTA-uniform
        const double *W = scr.W(p);
        const int ldw = scr.nmax;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int k0 = i0; k0 < n; k0 += kTile) {
            __syncthreads();
            for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
                const int kk = e / kTile, cc = e % kTile;
                const int k = k0 + kk;
                Wi[kk][cc] = (k < n && i0 + cc < n) ? W[(size_t)k * ldw + i0 + cc] : 0.0;
                Wj[kk][cc] = (k < n && j0 + cc < n) ? W[(size_t)k * ldw + j0 + cc] : 0.0;
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < kTile; ++kk) {
                const double wj = Wj[kk][tx];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) acc[rr] += Wi[kk][ty + 8 * rr] * wj;
            }
        }
        const double *Qs = scr.Q(p), *QN = scr.QN(p);
        double *Pp = P + poff[p];
        const int j = j0 + tx;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr) {
            const int i = i0 + ty + 8 * rr;
            if (i >= n || j >= n || (I == J && j > i)) continue;
            double v = acc[rr];
            if (schur)
#pragma unroll
                for (int bb = 0; bb < 6; ++bb) v -= QN[6 * i + bb] * Qs[6 * j + bb];
            Pp[(size_t)i * m + j] = v;
            Pp[(size_t)j * m + i] = v;
        }
    }
}

// S3' for the factored form (instead of S3 and S4): P_p keeps L^T in its
// upper triangle (written by S2) and receives G = L^-1 K_p in the border
// columns n..n+5 of rows 0..n-1 and 1 / L_kk in the border row n; the corner
// already holds -N.  precond_apply_factored_kernel applies it.
__global__ void __launch_bounds__(256) pc_keep_factor_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    double *__restrict__ P, SplitScratch scr)
{
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    const int lane = threadIdx.x & 31;
    for (int64_t p = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < nb;
         p += warps) {
        const int n = 3 * (int)(start[p + 1] - start[p]), m = n + 6;
        double *Pp = P + poff[p];
        const double *G = scr.G(p), *dW = scr.dW(p);
        for (int i = lane; i < n; i += 32) {
#pragma unroll
            for (int b = 0; b < 6; ++b) Pp[(size_t)i * m + n + b] = G[6 * i + b];
            Pp[(size_t)n * m + i] = dW[i];
        }
    }
}

// Runs S1..S4 over groups of bodies whose scratch fits the cap (S1, S2, S3'
// with `factored`).
mb_status setup_split(mb_context *ctx, int64_t nb, const double *r, const double *q,
                      const int64_t *start, const int64_t *poff, double *P, int max_np, double a,
                      double eta, int wall, int *flag, int flag_slot, int schur, cudaStream_t s,
                      const double *shift, bool factored = false)
{
    const int nmax = 3 * max_np;
    const int64_t stride = split_stride(nmax);
    const int64_t cap_bytes = (int64_t)MB_SETUP_SCRATCH_MB << 20;
    const int64_t group = std::max<int64_t>(1, std::min<int64_t>(nb, cap_bytes / (8 * stride)));
    MB_TRY(ensure(ctx, ctx->sol_dots, sizeof(double) * stride * group, "preconditioner scratch"));
    SplitScratch scr{(double *)ctx->sol_dots.ptr, stride, nmax};
    const PairConsts<double> k = PairConsts<double>::make(a);
    const double scale = 1.0 / (6.0 * 3.14159265358979323846 * eta * a);
    const bool lsmem = nmax <= kSmemMaxRows;
    const size_t fsmem =
        sizeof(double) * (lsmem ? (size_t)nmax * nmax + (7 + kPanel) * (size_t)nmax + 72
                                : 2 * (size_t)nmax + 72);
    const int col_groups = (int)ceil_div(nmax, 8);
    const int T = (int)ceil_div(nmax, kTile);
    const int tiles = T * (T + 1) / 2;
    for (int64_t g0 = 0; g0 < nb; g0 += group) {
        const int64_t ng = std::min(group, nb - g0);
        const int64_t *st = start + g0;
        const int64_t *po = poff + g0;
        const dim3 ga((unsigned)std::min<int64_t>(ceil_div(ng * max_np, 2), 32 * (int64_t)ctx->sm_count),
                      (unsigned)ceil_div(max_np, 32));
        if (wall)
            pc_assemble_kernel<true><<<ga, 64, 0, s>>>(ng, r, st, po, k, scale, P, shift);
        else
            pc_assemble_kernel<false><<<ga, 64, 0, s>>>(ng, r, st, po, k, scale, P, shift);
        if (ng < ctx->sm_count) {
            // fewer bodies than SMs: a cluster of CTAs per body, the rows in
            // shared memory or in place in global memory
            const size_t csm = factor_cluster_smem(nmax, lsmem);
            auto fk = lsmem ? pc_factor_cluster_kernel<true> : pc_factor_cluster_kernel<false>;
            MB_CUDA_TRY(ctx, cudaFuncSetAttribute(fk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)csm));
            fk<<<(int)ng * kFacCluster, 256, csm, s>>>(ng, r, q + 3 * g0, st, po, P, scr, flag,
                                                       flag_slot, g0, schur);
        } else {
            auto factor = lsmem ? pc_factor_kernel<true> : pc_factor_kernel<false>;
            MB_CUDA_TRY(ctx, cudaFuncSetAttribute(factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)fsmem));
            factor<<<(int)std::min<int64_t>(ng, 4 * (int64_t)ctx->sm_count), 256, fsmem, s>>>(
                ng, r, q + 3 * g0, st, po, P, scr, flag, flag_slot, g0, schur);
        }
        if (factored) {
            pc_keep_factor_kernel<<<(int)std::min<int64_t>(ceil_div(ng, 8), 8 * (int64_t)ctx->sm_count),
                                    256, 0, s>>>(ng, st, po, P, scr);
            count_launch(3);
            MB_CUDA_TRY(ctx, cudaGetLastError());
            continue;
        }
        const int gt = (int)std::min<int64_t>(ng * col_groups, 16 * (int64_t)ctx->sm_count);
        if (nmax > kSplitMaxRows) {
            const size_t tsm = sizeof(double) * (size_t)nmax * kTrinvSmemWarps;
            MB_CUDA_TRY(ctx, cudaFuncSetAttribute(pc_trinv_smem_kernel,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)tsm));
            pc_trinv_smem_kernel<<<gt, 32 * kTrinvSmemWarps, tsm, s>>>(ng, st, po, P, scr,
                                                                      col_groups);
        } else if (nmax <= 4 * kTile) {
            // double-float S3 and S4 (see pc_to_df_kernel)
            const int gc = (int)std::min<int64_t>(ceil_div(ng * nmax, 8), 8 * (int64_t)ctx->sm_count);
            pc_to_df_kernel<<<gc, 256, 0, s>>>(ng, st, po, P, scr);
            if (ng < ctx->sm_count) {
                // four columns per CTA, a warp pair each; the staged triangle
                // of L^T, G and the pairs' exchange
                const int cg4 = (int)ceil_div(nmax, 4);
                const int gt4 = (int)std::min<int64_t>(ng * cg4, 16 * (int64_t)ctx->sm_count);
                const size_t tsm = sizeof(double) * ((size_t)nmax * (nmax - 1) / 2 + 6 * (size_t)nmax) +
                                   sizeof(dfl) * (4 * 2 * 32 + 4 * 6);
                MB_CUDA_TRY(ctx, cudaFuncSetAttribute(pc_trinv_df_pair_kernel,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)tsm));
                pc_trinv_df_pair_kernel<<<gt4, 256, tsm, s>>>(ng, st, po, P, scr, cg4);
                const int T16 = (int)ceil_div(nmax, 16), tiles16 = T16 * (T16 + 1) / 2;
                const int gp = (int)std::min<int64_t>(ng * tiles16, 16 * (int64_t)ctx->sm_count);
                pc_product_df_kernel<16><<<gp, 256, 0, s>>>(ng, st, po, P, scr, tiles16, schur);
            } else {
                pc_trinv_df_kernel<<<gt, 256, 0, s>>>(ng, st, po, P, scr, col_groups);
                const int gp = (int)std::min<int64_t>(ng * tiles, 16 * (int64_t)ctx->sm_count);
                pc_product_df_kernel<kTile><<<gp, 256, 0, s>>>(ng, st, po, P, scr, tiles, schur);
            }
            count_launch(5);
            MB_CUDA_TRY(ctx, cudaGetLastError());
            continue;
        } else if (nmax <= 256)
            pc_trinv_kernel<8><<<gt, 256, 0, s>>>(ng, st, po, P, scr, col_groups);
        else
            pc_trinv_kernel<16><<<gt, 256, 0, s>>>(ng, st, po, P, scr, col_groups);
        const int gp = (int)std::min<int64_t>(ng * tiles, 16 * (int64_t)ctx->sm_count);
        pc_product_kernel<<<gp, 256, 0, s>>>(ng, st, po, P, scr, tiles, schur);
        count_launch(4);
        MB_CUDA_TRY(ctx, cudaGetLastError());
    }
    return MB_OK;
}

// Shared unbounded-domain preconditioner (MB_PRECOND_FREE_SHARED).  The
// free-space block of a body rotated by R is R~ M_ref R~^T, R~ = diag(R, ..,
// R), and K_p = R~ K_ref diag(R^T, R^T) blob by blob (K_ref from the
// reference offsets), so the whole indefinite block inverse is
// diag(R~, R, R) P_ref^-1 diag(R~, R, R)^T (Section 2.2.2).  Work items are
// (body, chunk of rows) like precond_apply_kernel; rows come in whole
// triples so that each CTA rotates its own results back.
__device__ __forceinline__ void quat_matrix(const double *__restrict__ th, double R[9])
{
    double s = th[0], x = th[1], y = th[2], z = th[3];
    const double inv = rsqrt(s * s + x * x + y * y + z * z);
    s *= inv; x *= inv; y *= inv; z *= inv;
    // R = (s^2 - v.v) I + 2 v v^T + 2 s [v]x
    const double d = s * s - (x * x + y * y + z * z);
    R[0] = d + 2.0 * x * x;     R[1] = 2.0 * x * y - 2.0 * s * z; R[2] = 2.0 * x * z + 2.0 * s * y;
    R[3] = 2.0 * y * x + 2.0 * s * z; R[4] = d + 2.0 * y * y;     R[5] = 2.0 * y * z - 2.0 * s * x;
    R[6] = 2.0 * z * x - 2.0 * s * y; R[7] = 2.0 * z * y + 2.0 * s * x; R[8] = d + 2.0 * z * z;
}

__global__ void __launch_bounds__(256) precond_apply_shared_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int *__restrict__ shape,
    const int64_t *__restrict__ poff, const double *__restrict__ P,
    const double *__restrict__ theta, const double *__restrict__ w, const double *__restrict__ g,
    double *__restrict__ lam, double *__restrict__ UO, int chunks, int rows, int body_rows)
{
    extern __shared__ double xs[];  // me rotated inputs, then `rows` results
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t item = blockIdx.x; item < nb * chunks; item += gridDim.x) {
        const int64_t p = item / chunks;
        const int r0 = (int)(item % chunks) * rows;
        const int64_t b0 = start[p];
        const int np = (int)(start[p + 1] - b0), n = 3 * np, m = n + 6, me = n + body_rows;
        const int r1 = min(me, r0 + rows);
        if (r0 >= me) continue;  // uniform over the CTA
        double R[9];
        quat_matrix(theta + 4 * p, R);
        double *ys = xs + me;
        __syncthreads();
        // x = diag(R~, R, R)^T [w_p; g_p], one triple per thread
        for (int t = threadIdx.x; t < me / 3; t += blockDim.x) {
            const double *v = t < np ? w + 3 * (b0 + t) : g + 6 * p + 3 * (t - np);
#pragma unroll
            for (int al = 0; al < 3; ++al)
                xs[3 * t + al] = R[al] * v[0] + R[3 + al] * v[1] + R[6 + al] * v[2];
        }
        __syncthreads();
        const double *Pp = P + poff[shape[p]];
        for (int row = r0 + warp; row < r1; row += nw) {
            const double *pr = Pp + (size_t)row * m;
            double acc = 0.0;
            for (int c = lane; c < me; c += 32) acc += pr[c] * xs[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) ys[row - r0] = acc;
        }
        __syncthreads();
        // rotate the triples of this chunk back
        for (int t = r0 / 3 + threadIdx.x; t < r1 / 3; t += blockDim.x) {
            const double *y = ys + 3 * t - r0;
            double *out = t < np ? lam + 3 * (b0 + t) : UO + 6 * p + 3 * (t - np);
#pragma unroll
            for (int al = 0; al < 3; ++al)
                out[al] = R[3 * al] * y[0] + R[3 * al + 1] * y[1] + R[3 * al + 2] * y[2];
        }
    }
}

}  // namespace

mb_status precond_setup(mb_context *ctx, int64_t nb, int64_t n, const double *r,
                        const double *q, const int64_t *blob_start, double a, double eta,
                        int wall, cudaStream_t s, int schur, const double *shift)
{
    // body sizes on the host
    std::vector<int64_t> hstart(nb + 1);
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(hstart.data(), blob_start, sizeof(int64_t) * (nb + 1),
                                     cudaMemcpyDeviceToHost, s));
    MB_TRY(wait_stream(ctx, s, "preconditioner setup"));
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
    const size_t small = sizeof(double) * (13 * (size_t)nmax + 72);
    const size_t smem = small + (lsmem ? sizeof(double) * (size_t)nmax * nmax : 0);
    const PairConsts<double> k = PairConsts<double>::make(a);
    const double scale = 1.0 / (6.0 * 3.14159265358979323846 * eta * a);
    int grid = (int)std::min<int64_t>(nb, 4 * (int64_t)ctx->sm_count);
    double *scratch = nullptr;
    int64_t stride = 0;
    if (!lsmem && nmax > kSplitMaxRowsSmem) {
        grid = (int)std::min<int64_t>(nb, ctx->sm_count);
        stride = (int64_t)nmax * nmax;
        MB_TRY(ensure(ctx, ctx->sol_dots, sizeof(double) * stride * grid, "Cholesky scratch"));
        scratch = (double *)ctx->sol_dots.ptr;
    }
    // Many bodies with large blocks keep the factored form: its application
    // costs the FP64 FMAs of the explicit inverse's GEMV and its setup a third
    // of the explicit inverse's (no L^-1, no W^T W).  Few or small bodies keep
    // the explicit inverse, whose application spreads over many CTAs.
    const bool factored = !lsmem && nmax <= kSplitMaxRowsSmem && nb >= ctx->sm_count;
    auto launch = [&](auto kern) -> mb_status {
        if (nmax <= kSplitMaxRowsSmem)
            return setup_split(ctx, nb, r, q, (const int64_t *)ctx->blob_start_copy.ptr,
                               (const int64_t *)ctx->pinv_off.ptr, (double *)ctx->pinv.ptr, max_np,
                               a, eta, wall, (int *)ctx->flag.ptr, -1, schur, s, shift, factored);
        MB_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        kern<<<grid, kSetupThreads, smem, s>>>(nb, r, q, (const int64_t *)ctx->blob_start_copy.ptr,
                                               (const int64_t *)ctx->pinv_off.ptr, k, scale,
                                               (double *)ctx->pinv.ptr, scratch, stride,
                                               (int *)ctx->flag.ptr, -1, schur, shift);
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
    MB_TRY(wait_stream(ctx, s, "preconditioner setup"));
    ctx->pc_nb = nb;
    ctx->pc_n = n;
    ctx->pc_max_np = max_np;
    ctx->pc_doubles = off[nb];
    ctx->pc_f32_ready = false;
    ctx->pc_kind = MB_PRECOND_WALL;
    ctx->pc_shapes = 0;
    ctx->pc_schur = schur;
    ctx->pc_factored = factored ? 1 : 0;
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
                              cudaStream_t s, int schur)
{
    const int nmax = 3 * max_np;
    const bool lsmem = nmax <= kSmemMaxRows;
    const size_t small = sizeof(double) * (13 * (size_t)nmax + 72);
    const size_t smem = small + (lsmem ? sizeof(double) * (size_t)nmax * nmax : 0);
    const PairConsts<double> k = PairConsts<double>::make(a);
    const double scale = 1.0 / (6.0 * 3.14159265358979323846 * eta * a);
    int grid = (int)std::min<int64_t>(nb, 4 * (int64_t)ctx->sm_count);
    double *scratch = nullptr;
    int64_t stride = 0;
    if (!lsmem && nmax > kSplitMaxRowsSmem) {
        grid = (int)std::min<int64_t>(nb, ctx->sm_count);
        stride = (int64_t)nmax * nmax;
        MB_TRY(ensure(ctx, ctx->sol_dots, sizeof(double) * stride * grid, "Cholesky scratch"));
        scratch = (double *)ctx->sol_dots.ptr;
    }
    auto launch = [&](auto kern) -> mb_status {
        if (nmax <= kSplitMaxRowsSmem)
            return setup_split(ctx, nb, r, q, start, poff, P, max_np, a, eta, wall, flags,
                               flag_slot, schur, s, nullptr);
        MB_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
        kern<<<grid, kSetupThreads, smem, s>>>(nb, r, q, start, poff, k, scale, P, scratch, stride,
                                               flags, flag_slot, schur, nullptr);
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

mb_status precond_setup_shared(mb_context *ctx, int64_t nb, int64_t n, const double *theta,
                               const int64_t *blob_start, const double *rho, double a,
                               double eta, cudaStream_t s, int schur)
{
    // offsets and reference positions on the host, to group bodies by shape
    std::vector<int64_t> hstart(nb + 1);
    std::vector<double> hrho(3 * (size_t)n);
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(hstart.data(), blob_start, sizeof(int64_t) * (nb + 1),
                                     cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(hrho.data(), rho, sizeof(double) * 3 * (size_t)n,
                                     cudaMemcpyDeviceToHost, s));
    MB_TRY(wait_stream(ctx, s, "preconditioner setup"));
    if (hstart[0] != 0 || hstart[nb] != n)
        return set_err(ctx, MB_EINVAL, "blob_start[0] must be 0 and blob_start[n_b] = N");
    // shape of every body: bodies with the same blob count and bitwise equal
    // offsets share one (an FNV-style hash over the 64-bit words, confirmed
    // by comparison)
    std::vector<int> shape(nb);
    std::vector<int64_t> rep_body;                 // first body of each shape
    std::unordered_map<uint64_t, std::vector<int>> by_hash;
    int max_np = 0;
    for (int64_t p = 0; p < nb; ++p) {
        const int64_t np = hstart[p + 1] - hstart[p];
        if (np < 1) return set_err(ctx, MB_EINVAL, "body %lld has no blobs", (long long)p);
        max_np = std::max<int>(max_np, (int)np);
        uint64_t h = 1469598103934665603ull ^ (uint64_t)np;
        for (int64_t e = 3 * hstart[p]; e < 3 * hstart[p + 1]; ++e) {
            uint64_t bits;
            std::memcpy(&bits, &hrho[e], sizeof(bits));
            h = (h ^ bits) * 1099511628211ull;
            h ^= h >> 29;
        }
        int found = -1;
        for (int t : by_hash[h]) {
            const int64_t q0 = rep_body[t];
            if (hstart[q0 + 1] - hstart[q0] == np &&
                std::memcmp(hrho.data() + 3 * hstart[q0], hrho.data() + 3 * hstart[p],
                            sizeof(double) * 3 * (size_t)np) == 0) {
                found = t;
                break;
            }
        }
        if (found < 0) {
            found = (int)rep_body.size();
            rep_body.push_back(p);
            by_hash[h].push_back(found);
        }
        shape[p] = found;
    }
    const int64_t ns = (int64_t)rep_body.size();
    // reference bodies: positions rho, centre 0, identity orientation
    std::vector<int64_t> rstart(ns + 1), off(ns + 1);
    rstart[0] = 0;
    off[0] = 0;
    for (int64_t t = 0; t < ns; ++t) {
        const int64_t np = hstart[rep_body[t] + 1] - hstart[rep_body[t]];
        rstart[t + 1] = rstart[t] + np;
        off[t + 1] = off[t] + (3 * np + 6) * (3 * np + 6);
    }
    std::vector<double> ref(3 * (size_t)rstart[ns] + 3 * (size_t)ns, 0.0);
    for (int64_t t = 0; t < ns; ++t)
        std::memcpy(ref.data() + 3 * rstart[t], hrho.data() + 3 * hstart[rep_body[t]],
                    sizeof(double) * 3 * (size_t)(rstart[t + 1] - rstart[t]));
    const size_t ref_doubles = ref.size();
    MB_TRY(ensure(ctx, ctx->pc_ref, sizeof(double) * ref_doubles + sizeof(int64_t) * 2 * (ns + 1),
                  "preconditioner reference bodies"));
    MB_TRY(ensure(ctx, ctx->pinv, sizeof(double) * off[ns], "preconditioner"));
    MB_TRY(ensure(ctx, ctx->pinv_off, sizeof(int64_t) * (ns + 1), "preconditioner"));
    MB_TRY(ensure(ctx, ctx->blob_start_copy, sizeof(int64_t) * (nb + 1), "preconditioner"));
    MB_TRY(ensure(ctx, ctx->pc_type, sizeof(int) * nb, "preconditioner shapes"));
    MB_TRY(ensure(ctx, ctx->pc_theta, sizeof(double) * 4 * nb, "preconditioner orientations"));
    MB_TRY(ensure(ctx, ctx->flag, sizeof(int) * 4, "flags"));
    double *dref = (double *)ctx->pc_ref.ptr;
    int64_t *dstart = (int64_t *)(dref + ref_doubles);
    int64_t *doff = dstart + (ns + 1);
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(dref, ref.data(), sizeof(double) * ref_doubles,
                                     cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(dstart, rstart.data(), sizeof(int64_t) * (ns + 1),
                                     cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * (ns + 1),
                                     cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinv_off.ptr, off.data(), sizeof(int64_t) * (ns + 1),
                                     cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->blob_start_copy.ptr, hstart.data(),
                                     sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pc_type.ptr, shape.data(), sizeof(int) * nb,
                                     cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pc_theta.ptr, theta, sizeof(double) * 4 * nb,
                                     cudaMemcpyDeviceToDevice, s));
    const int big = 0x7fffffff;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->flag.ptr, &big, sizeof(int), cudaMemcpyHostToDevice, s));
    int max_ref_np = 0;
    for (int64_t t = 0; t < ns; ++t)
        max_ref_np = std::max<int>(max_ref_np, (int)(rstart[t + 1] - rstart[t]));
    MB_TRY(precond_setup_range(ctx, ns, dref, dref + 3 * rstart[ns], dstart, doff,
                               (double *)ctx->pinv.ptr, max_ref_np, a, eta, 0,
                               (int *)ctx->flag.ptr, -1, s, schur));
    int first_bad = big;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(&first_bad, ctx->flag.ptr, sizeof(int),
                                     cudaMemcpyDeviceToHost, s));
    MB_TRY(wait_stream(ctx, s, "preconditioner setup"));
    ctx->pc_nb = nb;
    ctx->pc_n = n;
    ctx->pc_max_np = max_np;
    ctx->pc_kind = MB_PRECOND_FREE_SHARED;
    ctx->pc_doubles = 0;
    ctx->pc_f32_ready = false;
    ctx->pc_factored = 0;
    ctx->pc_shapes = ns;
    ctx->pc_schur = schur;
    if (first_bad != big) {
        ctx->pc_nb = 0;
        return set_err(ctx, MB_ESINGULAR,
                       "body %lld: free-space block of its shape or its Schur complement is not "
                       "positive definite", (long long)rep_body[first_bad]);
    }
    return MB_OK;
}

// Application of the factored form (see pc_keep_factor_kernel), one CTA per
// body, x = the body's rows in shared memory:
//   y = L^-1 w                  forward substitution by panels of kFacPanel
//                               rows: warp 0 solves the panel's triangle,
//                               then all threads subtract the panel's columns
//                               from the rows below (rows of L^T, coalesced);
//   U = -N (g + G^T y)          the body rows (skipped for the blob block alone);
//   lambda = L^-T (y + G U)     backward substitution by panels from the
//                               bottom: the panel's rows first lose their dot
//                               products with the solved rows (a warp per
//                               row), then warp 0 solves the panel's triangle.
// The panel's triangle is staged in shared memory with its columns scaled by
// 1 / L_kk, so that each step of warp 0's dependent chain is one shuffle and
// one FMA.  The same FMAs as the explicit inverse's GEMV (n^2 per body).
constexpr int kFacPanel = 32;

__global__ void __launch_bounds__(256) precond_apply_factored_kernel(
    int64_t nb, const int64_t *__restrict__ start, const int64_t *__restrict__ poff,
    const double *__restrict__ P, const double *__restrict__ w, const double *__restrict__ g,
    double *__restrict__ lam, double *__restrict__ UO, int body_rows)
{
    extern __shared__ double x[];              // n: the body's vector
    __shared__ double T[kFacPanel * kFacPanel];  // scaled panel triangle
    __shared__ double red[8 * 6];
    __shared__ double hU[12];                   // h = g + G^T y, then U
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const unsigned full = 0xffffffffu;
    for (int64_t p = blockIdx.x; p < nb; p += gridDim.x) {
        const int64_t b0 = start[p];
        const int n = 3 * (int)(start[p + 1] - b0), m = n + 6;
        const double *Pp = P + poff[p];
        const double *dW = Pp + (size_t)n * m;  // border row n: 1 / L_kk
        __syncthreads();  // the previous body is finished with x, T, hU
        for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = w[3 * b0 + i];
        // ---- forward: y = L^-1 w; L[i][k] = Lt[k][i] = Pp[k m + i]
        for (int c0 = 0; c0 < n; c0 += kFacPanel) {
            const int pw = min(kFacPanel, n - c0);
            // T[k][l] = L[c0 + l][c0 + k] / L_kk for k < l (row k of L^T, scaled)
            for (int e = threadIdx.x; e < pw * pw; e += blockDim.x) {
                const int k = e / pw, l = e % pw;
                T[k * kFacPanel + l] = l > k ? Pp[(size_t)(c0 + k) * m + c0 + l] * dW[c0 + k] : 0.0;
            }
            __syncthreads();
            if (warp == 0) {
                // lane l: a = x[c0 + l] minus the panel's earlier columns;
                // y_k = a_k / L_kk at the end
                double a = lane < pw ? x[c0 + lane] : 0.0;
                for (int k = 0; k < pw - 1; ++k) {
                    const double ak = __shfl_sync(full, a, k);
                    if (lane > k) a -= T[k * kFacPanel + lane] * ak;
                }
                if (lane < pw) x[c0 + lane] = a * dW[c0 + lane];
            }
            __syncthreads();
            for (int i = c0 + pw + threadIdx.x; i < n; i += blockDim.x) {
                double s0 = x[i], s1 = 0.0, s2 = 0.0, s3 = 0.0;
                int k = 0;
                for (; k + 4 <= pw; k += 4) {
                    s0 -= Pp[(size_t)(c0 + k) * m + i] * x[c0 + k];
                    s1 -= Pp[(size_t)(c0 + k + 1) * m + i] * x[c0 + k + 1];
                    s2 -= Pp[(size_t)(c0 + k + 2) * m + i] * x[c0 + k + 2];
                    s3 -= Pp[(size_t)(c0 + k + 3) * m + i] * x[c0 + k + 3];
                }
                for (; k < pw; ++k) s0 -= Pp[(size_t)(c0 + k) * m + i] * x[c0 + k];
                x[i] = (s0 + s1) + (s2 + s3);
            }
            __syncthreads();
        }
        // ---- body rows: U = -N (g + G^T y); G[i][b] = Pp[i m + n + b]
        if (body_rows) {
            double hb[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const double yi = x[i];
#pragma unroll
                for (int b = 0; b < 6; ++b) hb[b] += Pp[(size_t)i * m + n + b] * yi;
            }
#pragma unroll
            for (int b = 0; b < 6; ++b) {
                double v = hb[b];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
                if (lane == 0) red[6 * warp + b] = v;
            }
            __syncthreads();
            if (threadIdx.x < 6) {
                double h = g[6 * p + threadIdx.x];
                for (int ww = 0; ww < nw; ++ww) h += red[6 * ww + threadIdx.x];
                hU[threadIdx.x] = h;
            }
            __syncthreads();
            if (threadIdx.x < 6) {
                // the corner holds -N
                double u = 0.0;
#pragma unroll
                for (int b = 0; b < 6; ++b) u += Pp[(size_t)(n + threadIdx.x) * m + n + b] * hU[b];
                hU[6 + threadIdx.x] = u;
                UO[6 * p + threadIdx.x] = u;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                double v = x[i];
#pragma unroll
                for (int b = 0; b < 6; ++b) v += Pp[(size_t)i * m + n + b] * hU[6 + b];
                x[i] = v;
            }
            __syncthreads();
        }
        // ---- backward: lambda = L^-T x; row k of L^T is Pp[k m + k ..]
        for (int c1 = n; c1 > 0; c1 -= kFacPanel) {
            const int c0 = c1 > kFacPanel ? c1 - kFacPanel : 0, pw = c1 - c0;
            // the panel's rows lose their products with the solved rows
            for (int k = warp; k < pw; k += nw) {
                const double *lr = Pp + (size_t)(c0 + k) * m;
                double sacc = 0.0;
                for (int i = c1 + lane; i < n; i += 32) sacc += lr[i] * x[i];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(full, sacc, o);
                if (lane == 0) x[c0 + k] -= sacc;
            }
            // T[l][k] = Lt[c0 + l][c0 + k] / L_kk for l < k
            for (int e = threadIdx.x; e < pw * pw; e += blockDim.x) {
                const int l = e / pw, k = e % pw;
                T[l * kFacPanel + k] = l < k ? Pp[(size_t)(c0 + l) * m + c0 + k] * dW[c0 + k] : 0.0;
            }
            __syncthreads();
            if (warp == 0) {
                double a = lane < pw ? x[c0 + lane] : 0.0;
                for (int k = pw - 1; k > 0; --k) {
                    const double ak = __shfl_sync(full, a, k);
                    if (lane < k) a -= T[lane * kFacPanel + k] * ak;
                }
                if (lane < pw) x[c0 + lane] = a * dW[c0 + lane];
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) lam[3 * b0 + i] = x[i];
    }
}

static void precond_apply_impl(mb_context *ctx, const double *w, const double *g, double *lam,
                               double *UO, cudaStream_t s, int body_rows = 6, bool f32 = false)
{
    const int m = 3 * ctx->pc_max_np + body_rows;
    // few bodies: split each body's rows so that about two CTAs per SM have work
    const int64_t want = ceil_div(2 * (int64_t)ctx->sm_count, ctx->pc_nb);
    const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(want, ceil_div(m, 8)));
    const int grid = (int)std::min<int64_t>(ctx->pc_nb * chunks, 8 * (int64_t)ctx->sm_count);
    if (ctx->pc_kind == MB_PRECOND_FREE_SHARED) {
        const int rows = 3 * (int)ceil_div(m / 3, chunks);  // whole triples
        precond_apply_shared_kernel<<<grid, 256, sizeof(double) * (m + rows), s>>>(
            ctx->pc_nb, (const int64_t *)ctx->blob_start_copy.ptr, (const int *)ctx->pc_type.ptr,
            (const int64_t *)ctx->pinv_off.ptr, (const double *)ctx->pinv.ptr,
            (const double *)ctx->pc_theta.ptr, w, g, lam, UO, chunks, rows, body_rows);
        count_launch();
        return;
    }
    if (ctx->pc_factored) {
        const int gf = (int)std::min<int64_t>(ctx->pc_nb, 8 * (int64_t)ctx->sm_count);
        precond_apply_factored_kernel<<<gf, 256, sizeof(double) * 3 * ctx->pc_max_np, s>>>(
            ctx->pc_nb, (const int64_t *)ctx->blob_start_copy.ptr,
            (const int64_t *)ctx->pinv_off.ptr, (const double *)ctx->pinv.ptr, w, g, lam, UO,
            body_rows);
        count_launch();
        return;
    }
    const int rows = (int)ceil_div(m, chunks);
    if (f32)
        precond_apply_kernel<float><<<grid, 256, sizeof(float) * m, s>>>(
            ctx->pc_nb, (const int64_t *)ctx->blob_start_copy.ptr,
            (const int64_t *)ctx->pinv_off.ptr, (const float *)ctx->pinv32.ptr, w, g, lam, UO,
            chunks, rows, body_rows);
    else
        precond_apply_kernel<double><<<grid, 256, sizeof(double) * m, s>>>(
            ctx->pc_nb, (const int64_t *)ctx->blob_start_copy.ptr,
            (const int64_t *)ctx->pinv_off.ptr, (const double *)ctx->pinv.ptr, w, g, lam, UO,
            chunks, rows, body_rows);
    count_launch();
}

void precond_apply_packed(mb_context *ctx, const double *v, double *z, cudaStream_t s, bool f32)
{
    const int64_t n3 = 3 * ctx->pc_n;
    precond_apply_impl(ctx, v, v + n3, z, z + n3, s, 6, f32 && ctx->pc_f32_ready);
}

// The FP32 copy of the explicit wall blocks (precond_apply_packed with
// f32), for the FP32 inner iterations; does nothing for the other kinds.
mb_status precond_make_f32(mb_context *ctx, cudaStream_t s)
{
    ctx->pc_f32_ready = false;
    if (ctx->pc_nb == 0 || ctx->pc_kind != MB_PRECOND_WALL || ctx->pc_factored || ctx->pc_doubles == 0)
        return MB_OK;
    MB_TRY(ensure(ctx, ctx->pinv32, sizeof(float) * (size_t)ctx->pc_doubles, "FP32 preconditioner"));
    const int grid = (int)std::min<int64_t>(ceil_div(ctx->pc_doubles, 256), 8 * (int64_t)ctx->sm_count);
    pc_to_f32_kernel<<<grid, 256, 0, s>>>((const double *)ctx->pinv.ptr, ctx->pc_doubles,
                                          (float *)ctx->pinv32.ptr);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    ctx->pc_f32_ready = true;
    return MB_OK;
}

void precond_apply_blobs(mb_context *ctx, const double *w, double *z, cudaStream_t s)
{
    precond_apply_impl(ctx, w, nullptr, z, nullptr, s, 0);
}

mb_status precond_apply_public(mb_context *ctx, const double *w, const double *g, double *lam,
                               double *UO, cudaStream_t s)
{
    if (ctx->pc_nb == 0) return set_err(ctx, MB_EINVAL, "no preconditioner has been set up");
    if (!ctx->pc_schur)
        return set_err(ctx, MB_EINVAL, "the current blocks belong to a resistance solve; "
                                       "call mb_precond_setup again");
    if (3 * ctx->pc_max_np + 6 > 6000)
        return set_err(ctx, MB_EINVAL, "body too large for the preconditioner apply");
    precond_apply_impl(ctx, w, g, lam, UO, s);
    MB_CUDA_TRY(ctx, cudaGetLastError());
    return MB_OK;
}

}  // namespace mb
