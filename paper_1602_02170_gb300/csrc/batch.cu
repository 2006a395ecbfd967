// Batched mobility solves: many independent suspensions per launch
// (mb_solve_batch).
//
// The problems are concatenated on the device: blobs, bodies and the Krylov
// vectors use one global layout x = [lambda_all (3 N_tot) | (U, Omega) of
// every body (6 n_b,tot)], so the blob build, K, K^T and the block-diagonal
// preconditioner (Section 2.2.2; its blocks never couple bodies) run over
// all problems in one launch each.  The pair kernel runs as one persistent
// launch over a work list of (problem, target block, source chunk) items and
// couples blobs of the same problem only.  GMRES runs in lockstep: every
// problem owns its Hessenberg matrix and Givens rotations, dot products are
// segmented per problem, and a problem whose residual estimate reaches its
// target parks until the cycle ends; converged problems drop out of the work
// list, so their O(N^2) work stops.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "mb_internal.cuh"
#include "pair_tiles.cuh"

namespace mb {
namespace {

#ifndef MB_PAIR_NT
#define MB_PAIR_NT 256
#endif
constexpr int kNT = MB_PAIR_NT;
constexpr double kPi = 3.14159265358979323846;
constexpr int kRedChunk = 4096;   // elements per segmented-reduction item
constexpr int kRedThreads = 256;

struct ProbDesc {
    const double *q, *theta, *rho, *F, *T, *slip;
    const int64_t *blob_start;
    double *U, *Omega, *lambda;
    int64_t n, nb, blob_off, body_off;
};

struct BPlan {          // pair-kernel plan of one problem
    int64_t blob_off, n, chunk, item_off, part_off;
    int n_tblocks, S;
};

struct RedItem {        // one chunk of one problem's vector segment
    int64_t start, end;
    int prob;
};

// ------------------------------------------------------------------ layout
__global__ void concat_kernel(const ProbDesc *__restrict__ P, int np, double *rho_all,
                              double *q_all, double *theta_all, int64_t *start_all, double *F_all,
                              double *T_all, double *slip_all, int *blob_prob, int *body_prob,
                              int *flag)
{
    for (int p = blockIdx.x; p < np; p += gridDim.x) {
        const ProbDesc d = P[p];
        if (threadIdx.x == 0 && (d.blob_start[0] != 0 || d.blob_start[d.nb] != d.n))
            atomicMin(flag, p);
        for (int64_t e = threadIdx.x; e < 3 * d.n; e += blockDim.x) {
            rho_all[3 * d.blob_off + e] = d.rho[e];
            slip_all[3 * d.blob_off + e] = d.slip ? d.slip[e] : 0.0;
        }
        for (int64_t e = threadIdx.x; e < d.n; e += blockDim.x) blob_prob[d.blob_off + e] = p;
        for (int64_t e = threadIdx.x; e < d.nb; e += blockDim.x) {
            const int64_t b = d.body_off + e;
            for (int c = 0; c < 3; ++c) {
                q_all[3 * b + c] = d.q[3 * e + c];
                F_all[3 * b + c] = d.F[3 * e + c];
                T_all[3 * b + c] = d.T[3 * e + c];
            }
            for (int c = 0; c < 4; ++c) theta_all[4 * b + c] = d.theta[4 * e + c];
            body_prob[b] = p;
            // clamp keeps a malformed descriptor inside the problem's range
            int64_t s0 = d.blob_start[e];
            s0 = s0 < 0 ? 0 : (s0 > d.n ? d.n : s0);
            start_all[b] = d.blob_off + s0;
        }
    }
}

__global__ void scatter_solution_kernel(const ProbDesc *__restrict__ P, int np, int64_t n_tot,
                                        const double *__restrict__ x)
{
    for (int p = blockIdx.x; p < np; p += gridDim.x) {
        const ProbDesc d = P[p];
        for (int64_t e = threadIdx.x; e < 3 * d.n; e += blockDim.x)
            d.lambda[e] = x[3 * d.blob_off + e];
        for (int64_t e = threadIdx.x; e < 6 * d.nb; e += blockDim.x) {
            const int64_t b = e / 6, c = e % 6;
            const double v = x[3 * n_tot + 6 * d.body_off + e];
            if (c < 3) d.U[3 * b + c] = v;
            else d.Omega[3 * b + c - 3] = v;
        }
    }
}

__device__ __forceinline__ int find_item_owner(const int64_t *__restrict__ off, int np, int64_t item)
{
    int lo = 0, hi = np;  // off[lo] <= item < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ pair kernels
template <bool WALL, int NP>
__global__ void __launch_bounds__(kNT, NP == 1 ? 3 : 2) batch_x2_kernel(
    const BPlan *__restrict__ plans, const int64_t *__restrict__ item_off, int np,
    int64_t n_items, const int *__restrict__ mask, const float4 *__restrict__ hi,
    const float4 *__restrict__ lo, const double *__restrict__ f, double *__restrict__ y,
    double *__restrict__ partial, PairConsts2 k, double scale)
{
    __shared__ float4 sP[kX2SmemFloat4PerSource * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int p = find_item_owner(item_off, np, item);
        if (!mask[p]) continue;  // uniform across the CTA
        const BPlan P = plans[p];
        const int64_t local = item - P.item_off;
        const int tb = (int)(local % P.n_tblocks);
        const int64_t sc = local / P.n_tblocks;
        const int64_t j_begin = sc * P.chunk;
        const int64_t j_end = j_begin + P.chunk < P.n ? j_begin + P.chunk : P.n;
        double *out = P.S == 1 ? y + 3 * P.blob_off : partial + P.part_off + 3 * sc * P.n;
        x2_item<WALL, NP, kNT>(sP, hi + P.blob_off, lo + P.blob_off, f + 3 * P.blob_off, P.n, tb,
                               j_begin, j_end, k, out, P.S == 1 ? scale : 1.0);
    }
}

template <bool WALL>
__global__ void __launch_bounds__(kNT) batch_f64_kernel(
    const BPlan *__restrict__ plans, const int64_t *__restrict__ item_off, int np,
    int64_t n_items, const int *__restrict__ mask, const double *__restrict__ r,
    const double *__restrict__ f, double *__restrict__ y, double *__restrict__ partial,
    PairConsts<double> k, double scale)
{
    __shared__ double sm[6 * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int p = find_item_owner(item_off, np, item);
        if (!mask[p]) continue;
        const BPlan P = plans[p];
        const int64_t local = item - P.item_off;
        const int tb = (int)(local % P.n_tblocks);
        const int64_t sc = local / P.n_tblocks;
        const int64_t j_begin = sc * P.chunk;
        const int64_t j_end = j_begin + P.chunk < P.n ? j_begin + P.chunk : P.n;
        double *out = P.S == 1 ? y + 3 * P.blob_off : partial + P.part_off + 3 * sc * P.n;
        f64_item<WALL, kNT>(sm, r + 3 * P.blob_off, f + 3 * P.blob_off, P.n, tb, j_begin, j_end,
                            k, out, P.S == 1 ? scale : 1.0);
    }
}

template <bool WALL>
__global__ void __launch_bounds__(kNT) batch_df_kernel(
    const BPlan *__restrict__ plans, const int64_t *__restrict__ item_off, int np,
    int64_t n_items, const int *__restrict__ mask, const float4 *__restrict__ hi,
    const float4 *__restrict__ lo, const double *__restrict__ f, double *__restrict__ y,
    double *__restrict__ partial, PairConsts<dfl> k, double scale)
{
    __shared__ float4 sD[3 * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int p = find_item_owner(item_off, np, item);
        if (!mask[p]) continue;
        const BPlan P = plans[p];
        const int64_t local = item - P.item_off;
        const int tb = (int)(local % P.n_tblocks);
        const int64_t sc = local / P.n_tblocks;
        const int64_t j_begin = sc * P.chunk;
        const int64_t j_end = j_begin + P.chunk < P.n ? j_begin + P.chunk : P.n;
        double *out = P.S == 1 ? y + 3 * P.blob_off : partial + P.part_off + 3 * sc * P.n;
        df_item<WALL, kNT>(sD, hi + P.blob_off, lo + P.blob_off, f + 3 * P.blob_off, P.n, tb,
                           j_begin, j_end, k, out, P.S == 1 ? scale : 1.0);
    }
}

// y_i = scale * sum_s partial[s][i] for blobs of masked-in problems with S > 1
__global__ void batch_reduce_kernel(const BPlan *__restrict__ plans, const int *__restrict__ blob_prob,
                                    const int *__restrict__ mask, int64_t n_tot,
                                    const double *__restrict__ partial, double scale,
                                    double *__restrict__ y)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n_tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = blob_prob[e / 3];
        if (!mask[p]) continue;
        const BPlan P = plans[p];
        if (P.S == 1) continue;
        const int64_t loc = e - 3 * P.blob_off;
        double acc = 0.0;
        for (int s = 0; s < P.S; ++s) acc += partial[P.part_off + 3 * s * P.n + loc];
        y[e] = scale * acc;
    }
}

// ------------------------------------------------------------------ Krylov kernels
__device__ __forceinline__ int elem_prob(int64_t e, int64_t n_tot, const int *__restrict__ blob_prob,
                                         const int *__restrict__ body_prob)
{
    return e < 3 * n_tot ? blob_prob[e / 3] : body_prob[(e - 3 * n_tot) / 6];
}

// partial[k * n_items + it] = V[k] . w over reduction item it (masked problems only)
__global__ void batch_multidot_kernel(const double *__restrict__ V, int64_t ld, int nk,
                                      const double *__restrict__ w, const RedItem *__restrict__ items,
                                      int n_items, const int *__restrict__ mask,
                                      double *__restrict__ partial)
{
    __shared__ double red[kRedThreads / 32];
    const int k = blockIdx.y;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const RedItem I = items[it];
        double acc = 0.0;
        if (mask[I.prob]) {
            const double *v = V + (int64_t)k * ld;
            for (int64_t e = I.start + threadIdx.x; e < I.end; e += blockDim.x) acc += v[e] * w[e];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            acc = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (threadIdx.x == 0) partial[(int64_t)k * n_items + it] = acc;
        }
    }
}

// out[p*stride + k] = sum of problem p's items (fixed order), for k < nk
__global__ void batch_finish_dots_kernel(const double *__restrict__ partial, int n_items, int nk,
                                         const int *__restrict__ red_off, int np,
                                         const int *__restrict__ mask, double *__restrict__ out,
                                         int64_t stride)
{
    const int lane = threadIdx.x & 31;
    const int warps = (blockDim.x >> 5) * gridDim.x;
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < np * nk; w += warps) {
        const int p = w / nk, k = w % nk;
        if (!mask[p]) continue;
        double acc = 0.0;
        for (int it = red_off[p] + lane; it < red_off[p + 1]; it += 32)
            acc += partial[(int64_t)k * n_items + it];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) out[(int64_t)p * stride + k] = acc;
    }
}

// w -= sum_k V[k] h_p[k] (masked); h_p at sm + p*stride + h_off
__global__ void batch_subtract_span_kernel(const double *__restrict__ V, int64_t ld, int nk,
                                           const double *__restrict__ sm, int64_t stride,
                                           int64_t h_off, double *__restrict__ w, int64_t L,
                                           int64_t n_tot, const int *__restrict__ blob_prob,
                                           const int *__restrict__ body_prob,
                                           const int *__restrict__ mask)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = elem_prob(e, n_tot, blob_prob, body_prob);
        if (!mask[p]) continue;
        const double *h = sm + (int64_t)p * stride + h_off;
        double acc = w[e];
        for (int k = 0; k < nk; ++k) acc -= V[(int64_t)k * ld + e] * h[k];
        w[e] = acc;
    }
}

// y = x / sqrt(nrm2_p) (masked)
__global__ void batch_normalise_kernel(const double *x, double *y, int64_t L, const double *sm,
                                       int64_t stride, int64_t nrm_off, int64_t n_tot,
                                       const int *__restrict__ blob_prob,
                                       const int *__restrict__ body_prob,
                                       const int *__restrict__ mask)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = elem_prob(e, n_tot, blob_prob, body_prob);
        if (!mask[p]) continue;
        const double d = sqrt(sm[(int64_t)p * stride + nrm_off]);
        y[e] = d > 0.0 ? x[e] / d : 0.0;
    }
}

// x += sum_{k < kstep_p} Z[k] y_p[k]
__global__ void batch_add_span_kernel(const double *__restrict__ Z, int64_t ld,
                                      const double *__restrict__ sm, int64_t stride,
                                      int64_t y_off, const int *__restrict__ kstep,
                                      double *__restrict__ x, int64_t L, int64_t n_tot,
                                      const int *__restrict__ blob_prob,
                                      const int *__restrict__ body_prob)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int p = elem_prob(e, n_tot, blob_prob, body_prob);
        const int nk = kstep[p];
        if (nk == 0) continue;
        const double *y = sm + (int64_t)p * stride + y_off;
        double acc = x[e];
        for (int k = 0; k < nk; ++k) acc += Z[(int64_t)k * ld + e] * y[k];
        x[e] = acc;
    }
}

__global__ void sub_kernel(const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ z, int64_t L)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x)
        z[e] = a[e] - b[e];
}

__global__ void rhs_kernel(int64_t n, int64_t nb, const double *__restrict__ slip,
                           const double *__restrict__ F, const double *__restrict__ T,
                           double *__restrict__ b)
{
    const int64_t L = 3 * n + 6 * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < 3 * n) {
            b[e] = slip[e];
        } else {
            const int64_t k = e - 3 * n, p = k / 6, c = k % 6;
            b[e] = c < 3 ? -F[3 * p + c] : -T[3 * p + c - 3];
        }
    }
}

// Per-problem scalar layout (doubles), stride S.total():
//   H[(m+1) x m] column-major, cs[m], sn[m], g[m+1], y[m], h[m+1], nrm2, est,
//   bnorm, inner_abs, rel
struct BSmall {
    int m;
    __host__ __device__ int64_t H(int i, int j) const { return i + (int64_t)j * (m + 1); }
    __host__ __device__ int64_t cs() const { return (int64_t)(m + 1) * m; }
    __host__ __device__ int64_t sn() const { return cs() + m; }
    __host__ __device__ int64_t g() const { return sn() + m; }
    __host__ __device__ int64_t y() const { return g() + m + 1; }
    __host__ __device__ int64_t h() const { return y() + m; }
    __host__ __device__ int64_t nrm2() const { return h() + m + 1; }
    __host__ __device__ int64_t est() const { return nrm2() + 1; }
    __host__ __device__ int64_t bnorm() const { return est() + 1; }
    __host__ __device__ int64_t inner() const { return bnorm() + 1; }
    __host__ __device__ int64_t rel() const { return inner() + 1; }
    __host__ __device__ int64_t total() const { return rel() + 1; }
};

struct BState {        // per-problem integer state
    int *active;       // in the current Arnoldi cycle and not parked
    int *notdone;      // still being solved
    int *conv;         // converged
    int *kstep;        // Arnoldi steps taken in the current cycle
    int *iters;        // total Arnoldi steps
    int *restarts;     // completed cycles
    int *count;        // scratch counter (1 int)
};

__global__ void init_state_kernel(double *sm, BSmall B, BState st, int np)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        double *s = sm + (int64_t)p * B.total();
        s[B.bnorm()] = sqrt(s[B.nrm2()]);
        const bool zero = !(s[B.bnorm()] > 0.0);
        st.active[p] = 0;
        st.notdone[p] = zero ? 0 : 1;
        st.conv[p] = zero ? 1 : 0;
        st.kstep[p] = 0;
        st.iters[p] = 0;
        st.restarts[p] = 0;
        s[B.rel()] = 0.0;
    }
}

// After the true residual norms: decide done / start a new cycle.
__global__ void cycle_start_kernel(double *sm, BSmall B, BState st, int np, double tol,
                                   int maxit, int mixed)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        st.kstep[p] = 0;
        st.active[p] = 0;
        if (!st.notdone[p]) continue;
        double *s = sm + (int64_t)p * B.total();
        const double beta = sqrt(s[B.nrm2()]);
        const double rel = beta / s[B.bnorm()];
        s[B.rel()] = rel;
        if (rel <= tol) {
            st.conv[p] = 1;
            st.notdone[p] = 0;
            continue;
        }
        if (rel != rel || st.iters[p] >= maxit) {  // NaN residual or out of iterations
            st.notdone[p] = 0;
            continue;
        }
        for (int i = 0; i <= B.m; ++i) s[B.g() + i] = 0.0;
        s[B.g()] = beta;
        s[B.est()] = beta;
        double inner = 0.5 * tol * s[B.bnorm()];
        if (mixed) inner = fmax(inner, 1e-5 * beta);
        s[B.inner()] = inner;
        st.active[p] = 1;
        atomicAdd(st.count, 1);
    }
}

// Column j: merge the two CGS passes, rotate, update g; park converged problems.
__global__ void givens_kernel(double *sm, BSmall B, BState st, int np, int j, int maxit)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        if (!st.active[p]) continue;
        double *s = sm + (int64_t)p * B.total();
        for (int i = 0; i <= j; ++i) s[B.H(i, j)] = s[B.h() + i] + s[B.y() + i];
        s[B.H(j + 1, j)] = sqrt(s[B.nrm2()]);
        for (int i = 0; i < j; ++i) {
            const double c = s[B.cs() + i], sn = s[B.sn() + i];
            const double a = s[B.H(i, j)], b = s[B.H(i + 1, j)];
            s[B.H(i, j)] = c * a + sn * b;
            s[B.H(i + 1, j)] = -sn * a + c * b;
        }
        const double a = s[B.H(j, j)], b = s[B.H(j + 1, j)];
        const double rr = hypot(a, b);
        const double c = rr > 0.0 ? a / rr : 1.0;
        const double sn = rr > 0.0 ? b / rr : 0.0;
        s[B.cs() + j] = c;
        s[B.sn() + j] = sn;
        s[B.H(j, j)] = rr;
        s[B.H(j + 1, j)] = 0.0;
        const double gj = s[B.g() + j];
        s[B.g() + j] = c * gj;
        s[B.g() + j + 1] = -sn * gj;
        s[B.est()] = fabs(sn * gj);
        st.kstep[p] = j + 1;
        st.iters[p] += 1;
        if (!(s[B.est()] > s[B.inner()]) || st.iters[p] >= maxit || j + 1 >= B.m)
            st.active[p] = 0;  // parks until the cycle ends
        else
            atomicAdd(st.count, 1);
    }
}

__global__ void solve_triangles_kernel(double *sm, BSmall B, BState st, int np)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int k = st.kstep[p];
        if (k == 0) continue;
        double *s = sm + (int64_t)p * B.total();
        for (int i = k - 1; i >= 0; --i) {
            double acc = s[B.g() + i];
            for (int jj = i + 1; jj < k; ++jj) acc -= s[B.H(i, jj)] * s[B.y() + jj];
            const double d = s[B.H(i, i)];
            s[B.y() + i] = d != 0.0 ? acc / d : 0.0;
        }
        st.restarts[p] += 1;
    }
}

int vgrid(int64_t L) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 256), 4096)); }

}  // namespace

// ------------------------------------------------------------------ host driver
namespace {

struct Batch {
    mb_context *ctx;
    cudaStream_t s;
    int np;
    int64_t n_tot, nb_tot, L;
    double a, eta;
    int wall, m;
    BSmall B;
    BState st;
    // device arrays
    ProbDesc *desc;
    double *r, *rho, *q, *theta, *F, *T, *slip;
    int64_t *start;
    int *blob_prob, *body_prob;
    BPlan *plan32, *plan64;
    int64_t *item_off32, *item_off64;
    int64_t items32 = 0, items64 = 0;
    RedItem *red;
    int *red_off;
    int n_red = 0;
    double *partial;     // pair-kernel chunk partials
    double *dpart;       // reduction partials
    double *V, *Z, *b, *x, *w, *t, *sm;
    int grid32 = 0, grid64 = 0, np32 = 1;
    int *hcount;         // pinned

    mb_status matvec(const double *f, double *y, mb_precision prec, const int *mask)
    {
        const double scale = 1.0 / (6.0 * kPi * eta * a);
        if (prec == MB_DF64) {
            // the double-float kernel uses the FP64 kernel's plan (one target per thread)
            const float4 *hi = (const float4 *)ctx->pos_hi.ptr;
            const float4 *lo = (const float4 *)ctx->pos_lo.ptr;
            const PairConsts<dfl> k = PairConsts<dfl>::make(a);
            if (wall)
                batch_df_kernel<true><<<grid64, kNT, 0, s>>>(plan64, item_off64, np, items64, mask, hi,
                                                             lo, f, y, partial, k, scale);
            else
                batch_df_kernel<false><<<grid64, kNT, 0, s>>>(plan64, item_off64, np, items64, mask,
                                                              hi, lo, f, y, partial, k, scale);
            count_launch();
            batch_reduce_kernel<<<vgrid(3 * n_tot), 256, 0, s>>>(plan64, blob_prob, mask, n_tot,
                                                                 partial, scale, y);
            count_launch();
        } else if (prec == MB_FP64) {
            if (wall)
                batch_f64_kernel<true><<<grid64, kNT, 0, s>>>(plan64, item_off64, np, items64, mask, r,
                                                              f, y, partial, PairConsts<double>::make(a), scale);
            else
                batch_f64_kernel<false><<<grid64, kNT, 0, s>>>(plan64, item_off64, np, items64, mask,
                                                               r, f, y, partial, PairConsts<double>::make(a), scale);
            count_launch();
            batch_reduce_kernel<<<vgrid(3 * n_tot), 256, 0, s>>>(plan64, blob_prob, mask, n_tot,
                                                                 partial, scale, y);
            count_launch();
        } else {
            const float4 *hi = (const float4 *)ctx->pos_hi.ptr;
            const float4 *lo = (const float4 *)ctx->pos_lo.ptr;
            const PairConsts2 k = PairConsts2::make(a);
            auto *ev = profile_begin(ctx, s);
            if (np32 == 1) {
                if (wall)
                    batch_x2_kernel<true, 1><<<grid32, kNT, 0, s>>>(plan32, item_off32, np, items32, mask,
                                                                    hi, lo, f, y, partial, k, scale);
                else
                    batch_x2_kernel<false, 1><<<grid32, kNT, 0, s>>>(plan32, item_off32, np, items32,
                                                                     mask, hi, lo, f, y, partial, k, scale);
            } else {
                if (wall)
                    batch_x2_kernel<true, 2><<<grid32, kNT, 0, s>>>(plan32, item_off32, np, items32, mask,
                                                                    hi, lo, f, y, partial, k, scale);
                else
                    batch_x2_kernel<false, 2><<<grid32, kNT, 0, s>>>(plan32, item_off32, np, items32,
                                                                     mask, hi, lo, f, y, partial, k, scale);
            }
            profile_end(ev, s);
            count_launch();
            batch_reduce_kernel<<<vgrid(3 * n_tot), 256, 0, s>>>(plan32, blob_prob, mask, n_tot,
                                                                 partial, scale, y);
            count_launch();
        }
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }

    // y = A x for masked problems (other problems' rows are left arbitrary)
    mb_status apply_A(const double *xin, double *y, mb_precision prec, const int *mask)
    {
        MB_TRY(matvec(xin, y, prec, mask));
        launch_K_apply(nb_tot, n_tot, r, q, start, xin + 3 * n_tot, y, -1.0, 1.0, s);
        launch_KT_apply(nb_tot, r, q, start, xin, y + 3 * n_tot, -1.0, s);
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }

    void dots(const double *Vb, int nk, const double *wv, int64_t out_off, const int *mask)
    {
        const int gx = std::min(n_red, 4096);
        batch_multidot_kernel<<<dim3(gx, nk), kRedThreads, 0, s>>>(Vb, L, nk, wv, red, n_red, mask,
                                                                   dpart);
        count_launch();
        const int warps = np * nk;
        batch_finish_dots_kernel<<<(int)ceil_div(warps, 8), 256, 0, s>>>(
            dpart, n_red, nk, red_off, np, mask, sm + out_off, B.total());
        count_launch();
    }

    mb_status read_count(int *c)
    {
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(hcount, st.count, sizeof(int), cudaMemcpyDeviceToHost, s));
        MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        *c = *hcount;
        return MB_OK;
    }
    mb_status zero_count()
    {
        MB_CUDA_TRY(ctx, cudaMemsetAsync(st.count, 0, sizeof(int), s));
        return MB_OK;
    }
};

// Carve an aligned sub-buffer out of one workspace allocation.
struct Carver {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base + off);
        off += sizeof(T) * count;
        return p;
    }
};

}  // namespace

mb_status solve_batch(mb_context *ctx, int np, const mb_problem *probs, const mb_params *prm,
                      mb_info *infos, cudaStream_t s)
{
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    const int m = std::max(1, std::min(prm->restart, 500));
    Batch bt;
    bt.ctx = ctx; bt.s = s; bt.np = np; bt.a = prm->a; bt.eta = prm->eta; bt.wall = prm->wall;
    bt.m = m; bt.B = BSmall{m};

    // ---- host-side layout
    std::vector<ProbDesc> hd(np);
    int64_t n_tot = 0, nb_tot = 0;
    for (int p = 0; p < np; ++p) {
        const mb_problem &P = probs[p];
        hd[p] = ProbDesc{P.q, P.theta, P.rho, P.F, P.T, P.slip, P.blob_start, P.U, P.Omega,
                         P.lambda, P.n_blobs, P.n_bodies, n_tot, nb_tot};
        n_tot += P.n_blobs;
        nb_tot += P.n_bodies;
    }
    bt.n_tot = n_tot; bt.nb_tot = nb_tot; bt.L = 3 * n_tot + 6 * nb_tot;
    const int64_t L = bt.L;

    // pair-kernel plans: one chunk length for all problems, sized for ~8
    // items per resident CTA so that big and small problems balance
    int occ32 = 1, occ64 = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ32, batch_x2_kernel<true, 1>, kNT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ64, batch_f64_kernel<true>, kNT, 0);
    const int res32 = std::max(1, occ32) * ctx->sm_count, res64 = std::max(1, occ64) * ctx->sm_count;
    double pairs = 0.0;
    for (int p = 0; p < np; ++p) pairs += (double)hd[p].n * (double)hd[p].n;
    auto plan_for = [&](int tpc, int res, std::vector<BPlan> &pl, std::vector<int64_t> &ioff,
                        int64_t &items, int64_t &part) {
        const double per_item = pairs / (8.0 * res);
        int64_t chunk = (int64_t)std::ceil(per_item / tpc / kNT) * kNT;
        chunk = std::max<int64_t>(chunk, 2 * kNT);
        pl.resize(np);
        ioff.resize(np + 1);
        items = 0;
        part = 0;
        for (int p = 0; p < np; ++p) {
            BPlan b;
            b.blob_off = hd[p].blob_off;
            b.n = hd[p].n;
            b.n_tblocks = (int)ceil_div(b.n, tpc);
            b.S = (int)std::max<int64_t>(1, ceil_div(b.n, chunk));
            b.chunk = ceil_div(ceil_div(b.n, b.S), kNT) * kNT;
            b.S = (int)ceil_div(b.n, b.chunk);
            b.item_off = items;
            b.part_off = b.S > 1 ? part : 0;
            ioff[p] = items;
            items += (int64_t)b.n_tblocks * b.S;
            if (b.S > 1) part += 3 * b.n * b.S;
            pl[p] = b;
        }
        ioff[np] = items;
    };
    std::vector<BPlan> pl32, pl64;
    std::vector<int64_t> io32, io64;
    int64_t part32 = 0, part64 = 0;
    bt.np32 = 1;
    plan_for(2 * kNT, res32, pl32, io32, bt.items32, part32);
    plan_for(kNT, res64, pl64, io64, bt.items64, part64);
    bt.grid32 = (int)std::max<int64_t>(1, std::min<int64_t>(bt.items32, res32));
    bt.grid64 = (int)std::max<int64_t>(1, std::min<int64_t>(bt.items64, res64));

    // segmented-reduction items: each problem's blob and body segments in chunks
    std::vector<RedItem> red;
    std::vector<int> red_off(np + 1);
    for (int p = 0; p < np; ++p) {
        red_off[p] = (int)red.size();
        const int64_t segs[2][2] = {{3 * hd[p].blob_off, 3 * (hd[p].blob_off + hd[p].n)},
                                    {3 * n_tot + 6 * hd[p].body_off,
                                     3 * n_tot + 6 * (hd[p].body_off + hd[p].nb)}};
        for (auto &sg : segs)
            for (int64_t a0 = sg[0]; a0 < sg[1]; a0 += kRedChunk)
                red.push_back(RedItem{a0, std::min<int64_t>(sg[1], a0 + kRedChunk), p});
    }
    red_off[np] = (int)red.size();
    bt.n_red = (int)red.size();

    // ---- device workspace (one allocation, carved)
    const size_t need_misc =
        sizeof(ProbDesc) * np + sizeof(double) * (3 * n_tot * 3 + nb_tot * (3 + 4 + 3 + 3)) +
        sizeof(int64_t) * (nb_tot + 1) + sizeof(int) * (n_tot + nb_tot) +
        sizeof(BPlan) * 2 * np + sizeof(int64_t) * 2 * (np + 1) + sizeof(RedItem) * red.size() +
        sizeof(int) * (np + 1) + sizeof(int) * (6 * np + 1) +
        sizeof(double) * ((size_t)bt.B.total() * np + (size_t)(m + 1) * red.size()) + 64 * 256;
    const size_t need_vec = sizeof(double) * (size_t)L * (2 * m + 1 + 4);
    const size_t need_part = sizeof(double) * (size_t)std::max<int64_t>(1, std::max(part32, part64));
    MB_TRY(ensure(ctx, ctx->batch_ws, need_misc + need_vec + 64 * 256, "batch workspace"));
    MB_TRY(ensure(ctx, ctx->partial, need_part, "batch matvec partials"));
    MB_TRY(ensure(ctx, ctx->flag, sizeof(int) * 4, "flags"));
    if (!ctx->host_small) MB_CUDA_TRY(ctx, cudaMallocHost(&ctx->host_small, 64));
    bt.hcount = (int *)ctx->host_small;
    Carver cv{(char *)ctx->batch_ws.ptr};
    bt.desc = cv.take<ProbDesc>(np);
    bt.rho = cv.take<double>(3 * n_tot);
    bt.r = cv.take<double>(3 * n_tot);
    bt.slip = cv.take<double>(3 * n_tot);
    bt.q = cv.take<double>(3 * nb_tot);
    bt.theta = cv.take<double>(4 * nb_tot);
    bt.F = cv.take<double>(3 * nb_tot);
    bt.T = cv.take<double>(3 * nb_tot);
    bt.start = cv.take<int64_t>(nb_tot + 1);
    bt.blob_prob = cv.take<int>(n_tot);
    bt.body_prob = cv.take<int>(nb_tot);
    bt.plan32 = cv.take<BPlan>(np);
    bt.plan64 = cv.take<BPlan>(np);
    bt.item_off32 = cv.take<int64_t>(np + 1);
    bt.item_off64 = cv.take<int64_t>(np + 1);
    bt.red = cv.take<RedItem>(red.size());
    bt.red_off = cv.take<int>(np + 1);
    int *ints = cv.take<int>(6 * np + 1);
    bt.st = BState{ints, ints + np, ints + 2 * np, ints + 3 * np, ints + 4 * np, ints + 5 * np,
                   ints + 6 * np};
    bt.sm = cv.take<double>((size_t)bt.B.total() * np);
    bt.dpart = cv.take<double>((size_t)(m + 1) * red.size());
    bt.V = cv.take<double>((size_t)L * (m + 1));
    bt.Z = cv.take<double>((size_t)L * m);
    bt.b = cv.take<double>(L);
    bt.x = cv.take<double>(L);
    bt.w = cv.take<double>(L);
    bt.t = cv.take<double>(L);
    bt.partial = (double *)ctx->partial.ptr;

    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.desc, hd.data(), sizeof(ProbDesc) * np, cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.plan32, pl32.data(), sizeof(BPlan) * np, cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.plan64, pl64.data(), sizeof(BPlan) * np, cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.item_off32, io32.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.item_off64, io64.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.red, red.data(), sizeof(RedItem) * red.size(), cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.red_off, red_off.data(), sizeof(int) * (np + 1), cudaMemcpyHostToDevice, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.start + nb_tot, &n_tot, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    const int big = 0x7fffffff;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->flag.ptr, &big, sizeof(int), cudaMemcpyHostToDevice, s));
    concat_kernel<<<std::min(np, 4096), 256, 0, s>>>(bt.desc, np, bt.rho, bt.q, bt.theta, bt.start,
                                                     bt.F, bt.T, bt.slip, bt.blob_prob, bt.body_prob,
                                                     (int *)ctx->flag.ptr);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    int bad = big;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(&bad, ctx->flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (bad != big)
        return set_err(ctx, MB_EINVAL, "problem %d: blob_start[0] must be 0 and blob_start[n_b] = N", bad);

    // ---- blobs, preconditioner (all bodies of all problems at once)
    MB_TRY(blob_positions(ctx, nb_tot, n_tot, bt.q, bt.theta, bt.start, bt.rho, bt.r, s));
    {
        mb_status st = precond_setup(ctx, nb_tot, n_tot, bt.r, bt.q, bt.start, prm->a, prm->eta,
                                     prm->wall, s);
        if (st == MB_ESINGULAR) {
            // name the problem that owns the failing body
            const std::string msg = ctx->err;
            int body = -1;
            sscanf(msg.c_str(), "body %d", &body);
            int owner = -1;
            for (int p = 0; p < np && body >= 0; ++p)
                if (body >= hd[p].body_off && body < hd[p].body_off + hd[p].nb) owner = p;
            return set_err(ctx, MB_ESINGULAR, "problem %d, body %lld: mobility block not positive definite",
                           owner, owner >= 0 ? (long long)(body - hd[owner].body_off) : -1LL);
        }
        MB_TRY(st);
    }
    const bool use32 = prm->prec != MB_FP64;  // FP32 and double-float read packed positions
    if (use32) MB_TRY(matvec_pack_positions(ctx, bt.r, n_tot, s));
    MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const auto t1 = clk::now();

    const mb_precision inner = inner_precision(prm->prec);
    const mb_precision outer = outer_precision(prm->prec);
    const int vg = vgrid(L);
    const int pg = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(np, 128), 1024));
    const BSmall &B = bt.B;

    // autotune the packed-kernel shape (2 or 4 targets per thread) on the
    // first inner matvec of the batch: time both on all problems
    if (inner == MB_FP32_KAHAN) {
        std::vector<int> ones(np, 1);
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.st.notdone, ones.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
        float best = 1e30f;
        int best_np = 1;
        cudaEvent_t e0, e1;
        MB_CUDA_TRY(ctx, cudaEventCreate(&e0));
        MB_CUDA_TRY(ctx, cudaEventCreate(&e1));
        for (int cand = 1; cand <= 2; ++cand) {
            bt.np32 = cand;
            std::vector<BPlan> plc;
            std::vector<int64_t> ioc;
            int64_t itc = 0, ptc = 0;
            plan_for(2 * cand * kNT, res32, plc, ioc, itc, ptc);
            if ((size_t)ptc * sizeof(double) > ctx->partial.bytes) continue;
            MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.plan32, plc.data(), sizeof(BPlan) * np, cudaMemcpyHostToDevice, s));
            MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.item_off32, ioc.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, s));
            bt.items32 = itc;
            bt.grid32 = (int)std::max<int64_t>(1, std::min<int64_t>(itc, res32));
            MB_CUDA_TRY(ctx, cudaMemsetAsync(bt.x, 0, sizeof(double) * L, s));
            MB_CUDA_TRY(ctx, cudaEventRecord(e0, s));
            MB_TRY(bt.matvec(bt.x, bt.t, MB_FP32_KAHAN, bt.st.notdone));
            MB_CUDA_TRY(ctx, cudaEventRecord(e1, s));
            MB_CUDA_TRY(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            MB_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_np = cand; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        bt.np32 = best_np;
        std::vector<BPlan> plc;
        std::vector<int64_t> ioc;
        int64_t itc = 0, ptc = 0;
        plan_for(2 * best_np * kNT, res32, plc, ioc, itc, ptc);
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.plan32, plc.data(), sizeof(BPlan) * np, cudaMemcpyHostToDevice, s));
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.item_off32, ioc.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, s));
        bt.items32 = itc;
        bt.grid32 = (int)std::max<int64_t>(1, std::min<int64_t>(itc, res32));
    }

    // ---- rhs, norms, state
    rhs_kernel<<<vg, 256, 0, s>>>(n_tot, nb_tot, bt.slip, bt.F, bt.T, bt.b);
    count_launch();
    MB_CUDA_TRY(ctx, cudaMemsetAsync(bt.x, 0, sizeof(double) * L, s));
    {
        std::vector<int> ones(np, 1);
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.st.notdone, ones.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    }
    bt.dots(bt.b, 1, bt.b, B.nrm2(), bt.st.notdone);
    init_state_kernel<<<pg, 128, 0, s>>>(bt.sm, B, bt.st, np);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());

    bool first = true;
    for (int guard = 0; guard < 100000; ++guard) {
        // true residual w = b - A x for problems still being solved
        if (first) {
            MB_CUDA_TRY(ctx, cudaMemcpyAsync(bt.w, bt.b, sizeof(double) * L, cudaMemcpyDeviceToDevice, s));
            first = false;
        } else {
            MB_TRY(bt.apply_A(bt.x, bt.t, outer, bt.st.notdone));
            sub_kernel<<<vg, 256, 0, s>>>(bt.b, bt.t, bt.w, L);
            count_launch();
        }
        bt.dots(bt.w, 1, bt.w, B.nrm2(), bt.st.notdone);
        MB_TRY(bt.zero_count());
        cycle_start_kernel<<<pg, 128, 0, s>>>(bt.sm, B, bt.st, np, prm->tol, prm->maxit,
                                              prm->prec == MB_MIXED_REFINE);
        count_launch();
        int n_active = 0;
        MB_TRY(bt.read_count(&n_active));
        if (n_active == 0) break;
        batch_normalise_kernel<<<vg, 256, 0, s>>>(bt.w, bt.V, L, bt.sm, B.total(), B.nrm2(), n_tot,
                                                  bt.blob_prob, bt.body_prob, bt.st.active);
        count_launch();
        for (int j = 0; j < m; ++j) {
            double *vj = bt.V + (int64_t)j * L;
            double *zj = bt.Z + (int64_t)j * L;
            double *vn = bt.V + (int64_t)(j + 1) * L;
            precond_apply_packed(ctx, vj, zj, s);
            MB_TRY(bt.apply_A(zj, vn, inner, bt.st.active));
            bt.dots(bt.V, j + 1, vn, B.h(), bt.st.active);
            batch_subtract_span_kernel<<<vg, 256, 0, s>>>(bt.V, L, j + 1, bt.sm, B.total(), B.h(), vn,
                                                          L, n_tot, bt.blob_prob, bt.body_prob,
                                                          bt.st.active);
            count_launch();
            bt.dots(bt.V, j + 1, vn, B.y(), bt.st.active);
            batch_subtract_span_kernel<<<vg, 256, 0, s>>>(bt.V, L, j + 1, bt.sm, B.total(), B.y(), vn,
                                                          L, n_tot, bt.blob_prob, bt.body_prob,
                                                          bt.st.active);
            count_launch();
            bt.dots(vn, 1, vn, B.nrm2(), bt.st.active);
            batch_normalise_kernel<<<vg, 256, 0, s>>>(vn, vn, L, bt.sm, B.total(), B.nrm2(), n_tot,
                                                      bt.blob_prob, bt.body_prob, bt.st.active);
            count_launch();
            MB_TRY(bt.zero_count());
            givens_kernel<<<pg, 128, 0, s>>>(bt.sm, B, bt.st, np, j, prm->maxit);
            count_launch();
            MB_CUDA_TRY(ctx, cudaGetLastError());
            int still = 0;
            MB_TRY(bt.read_count(&still));
            if (still == 0) break;
        }
        solve_triangles_kernel<<<pg, 128, 0, s>>>(bt.sm, B, bt.st, np);
        count_launch();
        batch_add_span_kernel<<<vg, 256, 0, s>>>(bt.Z, L, bt.sm, B.total(), B.y(), bt.st.kstep, bt.x,
                                                 L, n_tot, bt.blob_prob, bt.body_prob);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
    }
    scatter_solution_kernel<<<std::min(np, 4096), 256, 0, s>>>(bt.desc, np, n_tot, bt.x);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());

    // per-problem results
    std::vector<int> conv(np), iters(np), restarts(np);
    std::vector<double> small((size_t)B.total() * np);
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(conv.data(), bt.st.conv, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(iters.data(), bt.st.iters, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(restarts.data(), bt.st.restarts, sizeof(int) * np, cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(small.data(), bt.sm, sizeof(double) * small.size(), cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const auto t2 = clk::now();
    const double setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    const double solve_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    int n_bad = 0;
    for (int p = 0; p < np; ++p) {
        if (!conv[p]) ++n_bad;
        if (infos) {
            infos[p].iters = iters[p];
            infos[p].restarts = restarts[p];
            infos[p].converged = conv[p];
            infos[p].rel_residual = small[(size_t)p * B.total() + B.rel()];
            infos[p].setup_ms = setup_ms;
            infos[p].solve_ms = solve_ms;
        }
    }
    if (n_bad)
        return set_err(ctx, MB_ENOTCONVERGED, "%d of %d problems did not converge within maxit", n_bad, np);
    return MB_OK;
}

}  // namespace mb
