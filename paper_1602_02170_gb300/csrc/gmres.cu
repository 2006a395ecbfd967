// Right-preconditioned flexible GMRES on the saddle-point system (Eq. saddle_M)
//     A [lambda; U] = [M lambda - K U; -K^T lambda] = [slip; -F]
// with the block-diagonal preconditioner of Section 2.2.2 (precond.cu).
//
// Vectors are packed as x = [lambda (3N) | (U, Omega) per body (6 n_b)] in
// FP64 and stay on the device.  Each Arnoldi step: z_j = P^-1 v_j, w = A z_j,
// classical Gram-Schmidt applied twice (CGS2), Givens rotations on the
// device.  The preconditioned vectors z_j are kept (flexible variant), so the
// update x += Z y is exact even when P^-1 or the inner matvec are inexact.
// Every restart recomputes the true residual b - A x; with MB_MIXED_REFINE
// the Arnoldi matvecs use the FP32 pair kernel and the restart residual a
// higher-precision one, which turns restarts into iterative refinement (the
// inexact-Krylov remark of Section 2.2.1).  Termination is on the true
// residual, as right preconditioning allows (Section 3.3.3, preconditioner
// discussion).
//
// Mixed precision keeps M lambda as an FP64 running sum y_M: each cycle's
// correction dx = Z y adds M dlambda to it, and A x = [y_M - K U; -K^T lambda]
// is rebuilt from y_M with the exact K / K^T kernels.  The correction of a
// cycle that started from a residual beta is about beta in size, so the FP32
// pair kernel's error on it (below ~1e-5 relative) is ~1e-5 beta: once
// beta <= kFineRel * tol * |b| that is under a tenth of the target and the
// increment runs in FP32; larger corrections (always the first one, which is
// the whole solution) run in double-float.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <cmath>
#include <vector>

#include <cooperative_groups.h>

#include "mb_internal.cuh"

namespace mb {
namespace {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;
// mixed precision: FP32 increments of y_M once the cycle's starting residual
// is below kFineRel * tol * |b| (see the header)
constexpr double kFineRel = 1e4;

int vec_grid(int64_t L) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(L, 256), 2048)); }

// partial[k * nblk + b] = sum over block b's slice of V[k] . w, for k < nk
__global__ void multidot_kernel(const double *__restrict__ V, int64_t ld, int nk,
                                const double *__restrict__ w, int64_t L, double *__restrict__ partial)
{
    __shared__ double red[kRedThreads / 32];
    const int k = blockIdx.y;
    const double *v = V + (int64_t)k * ld;
    double acc = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x)
        acc += v[e] * w[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (kRedThreads / 32) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partial[k * gridDim.x + blockIdx.x] = acc;
    }
}

// out[k] (+)= sum_b partial[k * nblk + b]; one warp per k, fixed order
__global__ void finish_dots_kernel(const double *__restrict__ partial, int nblk, int nk,
                                   double *__restrict__ out, int accumulate)
{
    const int k = blockIdx.x;
    if (k >= nk) return;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += 32) acc += partial[k * nblk + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[k] = accumulate ? out[k] + acc : acc;
}

// w -= sum_k V[k] h[k]
__global__ void subtract_span_kernel(const double *__restrict__ V, int64_t ld, int nk,
                                     const double *__restrict__ h, double *__restrict__ w, int64_t L)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        double acc = w[e];
        for (int k = 0; k < nk; ++k) acc -= V[(int64_t)k * ld + e] * h[k];
        w[e] = acc;
    }
}

// y = x / d with d = *denom (or sqrt(*denom)); y may alias x
__global__ void scale_kernel(const double *x, double *y, int64_t L, const double *denom,
                             int use_sqrt)
{
    double d = *denom;
    if (use_sqrt) d = sqrt(d);
    const double s = d > 0.0 ? 1.0 / d : 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = s * x[e];
}

// z = a - b
__global__ void sub_kernel(const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ z, int64_t L)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x)
        z[e] = a[e] - b[e];
}

// dx = sum_k Z[k] y[k]; x += dx
__global__ void update_span_kernel(const double *__restrict__ Z, int64_t ld, int nk,
                                   const double *__restrict__ y, double *__restrict__ x,
                                   double *__restrict__ dx, int64_t L)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < nk; ++k) acc += Z[(int64_t)k * ld + e] * y[k];
        dx[e] = acc;
        x[e] += acc;
    }
}

// y_M += t; t = y_M (first n3 entries)
__global__ void accumulate_kernel(double *__restrict__ t, double *__restrict__ ym, int64_t n3)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double v = ym[e] + t[e];
        ym[e] = v;
        t[e] = v;
    }
}

// x += sum_k Z[k] y[k]
__global__ void add_span_kernel(const double *__restrict__ Z, int64_t ld, int nk,
                                const double *__restrict__ y, double *__restrict__ x, int64_t L)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        double acc = x[e];
        for (int k = 0; k < nk; ++k) acc += Z[(int64_t)k * ld + e] * y[k];
        x[e] = acc;
    }
}

// Small Krylov state in one device array:
//   H[(m+1) x m] column-major (H[i + j*(m+1)]), cs[m], sn[m], g[m+1], y[m],
//   h[m+1] (current column), nrm2 (squared norm scratch), est
struct Small {
    int m;
    __host__ __device__ int64_t H(int i, int j) const { return i + (int64_t)j * (m + 1); }
    __host__ __device__ int64_t cs() const { return (int64_t)(m + 1) * m; }
    __host__ __device__ int64_t sn() const { return cs() + m; }
    __host__ __device__ int64_t g() const { return sn() + m; }
    __host__ __device__ int64_t y() const { return g() + m + 1; }
    __host__ __device__ int64_t h() const { return y() + m; }
    __host__ __device__ int64_t nrm2() const { return h() + m + 1; }
    __host__ __device__ int64_t est() const { return nrm2() + 1; }
    __host__ __device__ int64_t total() const { return est() + 1; }
};

// Start a cycle: g = [beta, 0, ...], beta = sqrt(nrm2); beta is posted like
// the Arnoldi steps' estimates (post: mapped host memory [value, count, step
// word]; a cycle start writes the first two, in FP64, behind a fence)
__global__ void cycle_start_kernel(double *__restrict__ sm, Small L, double *__restrict__ post,
                                   unsigned long long *__restrict__ seq)
{
    const double beta = sqrt(sm[L.nrm2()]);
    for (int i = 0; i <= L.m; ++i) sm[L.g() + i] = 0.0;
    sm[L.g()] = beta;
    sm[L.est()] = beta;
    if (post) {
        const unsigned long long q = *seq + 1;
        *seq = q;
        post[0] = beta;
        __threadfence_system();
        *(volatile unsigned long long *)(post + 1) = q;
    }
}

// The latest posted count in the mapped words [value, count, step word]: a
// cycle start's full count, or a later step's (its low 32 bits ahead of it).
static unsigned long long posted_count(const double *hp)
{
    const unsigned long long c1 = *(volatile const unsigned long long *)(hp + 1);
    const unsigned long long w = *(volatile const unsigned long long *)(hp + 2);
    const int32_t d = (int32_t)((uint32_t)(w >> 32) - (uint32_t)c1);
    return d > 0 ? c1 + (unsigned long long)d : c1;
}

// Column j of H is h[0..j] with H[j+1, j] = sqrt(nrm2); apply the previous
// rotations, form the new one and update g.  est = |g[j+1]|.
__device__ void givens_column(double *__restrict__ sm, Small L, int j)
{
    double col[2];
    for (int i = 0; i <= j; ++i) sm[L.H(i, j)] = sm[L.h() + i];
    const double hn = sqrt(sm[L.nrm2()]);
    sm[L.H(j + 1, j)] = hn;
    for (int i = 0; i < j; ++i) {
        const double c = sm[L.cs() + i], s = sm[L.sn() + i];
        col[0] = sm[L.H(i, j)];
        col[1] = sm[L.H(i + 1, j)];
        sm[L.H(i, j)] = c * col[0] + s * col[1];
        sm[L.H(i + 1, j)] = -s * col[0] + c * col[1];
    }
    const double a = sm[L.H(j, j)], b = sm[L.H(j + 1, j)];
    const double rr = hypot(a, b);
    const double c = rr > 0.0 ? a / rr : 1.0;
    const double s = rr > 0.0 ? b / rr : 0.0;
    sm[L.cs() + j] = c;
    sm[L.sn() + j] = s;
    sm[L.H(j, j)] = rr;
    sm[L.H(j + 1, j)] = 0.0;
    const double gj = sm[L.g() + j];
    sm[L.g() + j] = c * gj;
    sm[L.g() + j + 1] = -s * gj;
    sm[L.est()] = fabs(-s * gj);
}

__global__ void givens_kernel(double *__restrict__ sm, Small L, int j) { givens_column(sm, L, j); }

// Small systems: one launch does the whole orthogonalisation of w = V_{j+1}:
// both classical Gram-Schmidt passes (h = V^T w, w -= V h), their merged
// coefficients as column j of H, |w|, the Givens update and w /= |w|.  The
// same steps as the multi-kernel sequence, without its 9 launches.  T is the
// arithmetic of the passes: double, or float for the FP32 inner iterations
// of mixed precision, whose basis only needs FP32 orthogonality (the FP32
// matvec already limits the Arnoldi relation to that level, and the outer
// refinement restores FP64 accuracy).
constexpr int64_t kOrthSmallMax = 1 << 18;  // (j + 1) L up to this: one launch

// The launch is a cluster of kOrthCluster CTAs: CTA r owns the slice
// [r per, (r + 1) per) of every vector.  Each pass forms partial
// dot products over the slice, sums the kOrthCluster partials read from the
// other CTAs' shared memory (the same order in every CTA, so all hold the
// same coefficients) and updates its own slice.  Rank 0 does the Givens
// update.  On GB300 one SM sustains about 1.7 FP64 FMA per clock, so eight
// SMs shorten the FP64 passes; a cluster barrier costs a few hundred cycles.
constexpr int kOrthCluster = 8;
constexpr int kOrthClusterThreads = 256;
// A CTA's slices of V_0 .. V_{j+1} are staged in its shared memory when they
// take at most this many doubles (64 KB): all their loads are then in flight
// at once, and both passes, the norm and the scaling read shared memory
// instead of walking the slices through L2 one dependent round trip after
// another.  The arithmetic and its order are the same either way.
constexpr int64_t kOrthStageDoubles = 8192;

// 1/sqrt(d) in FP64: the FP32 estimate refined by one FP32 and two FP64
// Newton-Raphson steps, y <- y (3 - d y^2) / 2 (quadratic convergence: FP64
// accuracy).  FP64 instructions issue slowly on this chip, so this short
// sequence replaces the square roots and divisions of the serial parts of
// the orthogonalisation.  Arguments outside the FP32 range take 1 / sqrt.
__device__ __forceinline__ double rsqrt_fp64(double d)
{
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    const float df = (float)d;
    float yf = rsqrtf(df);
    yf = yf * (1.5f - 0.5f * df * yf * yf);
    double y = (double)yf;
    y = y * (1.5 - 0.5 * d * y * y);
    return y * (1.5 - 0.5 * d * y * y);
}

// The saddle operator's rows around M x (Eq. saddle_M) from the pair
// kernel's chunk partials, for the orthogonalisation to form w = A x itself
// instead of a separate launch: partial == nullptr when w is already formed.
struct SaddleIn {
    const double *partial = nullptr;  // S chunk partials of M x_lambda, 3n each
    int S = 0;
    double scale = 0.0;
    int64_t n = 0, nb = 0;
    const double *r = nullptr, *q = nullptr;
    const int64_t *start = nullptr;
    const int *body = nullptr;  // body of every blob (else found by bisection)
    const double *x = nullptr;  // [lambda; U]
};

// Row e of w = A x: blob rows scale sum_s partial[s][e] - (K U)_e (one
// thread each, the partials summed in four interleaved chains); body rows
// -(K^T lambda)_p,c
// (one warp each, lanes over the body's blobs).  Blob rows [b0, b1) are
// this CTA's; body rows are dealt to the warps of the whole cluster.
__device__ void saddle_rows_cluster(const SaddleIn &sd, double *__restrict__ w, int64_t b0,
                                    int64_t b1, int rank)
{
    const int64_t m3 = 3 * sd.n;
    for (int64_t e = b0 + threadIdx.x; e < b1 && e < m3; e += blockDim.x) {
        // four interleaved sums: a dependent FP64 add costs ~64 cycles here
        double a4[4] = {0.0, 0.0, 0.0, 0.0};
        int sc = 0;
        for (; sc + 4 <= sd.S; sc += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) a4[u] += sd.partial[(sc + u) * m3 + e];
        for (; sc < sd.S; ++sc) a4[0] += sd.partial[sc * m3 + e];
        const double acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
        const int64_t i = e / 3;
        const int c = (int)(e - 3 * i);
        const int64_t p = sd.body ? (int64_t)sd.body[i] : body_of(sd.start, sd.nb, i);
        const double dx = sd.r[3 * i] - sd.q[3 * p], dy = sd.r[3 * i + 1] - sd.q[3 * p + 1],
                     dz = sd.r[3 * i + 2] - sd.q[3 * p + 2];
        const double *u = sd.x + m3 + 6 * p;
        const double v = c == 0 ? u[0] + (u[4] * dz - u[5] * dy)
                       : c == 1 ? u[1] + (u[5] * dx - u[3] * dz)
                                : u[2] + (u[3] * dy - u[4] * dx);
        w[e] = __dsub_rn(__dmul_rn(sd.scale, acc), v);
    }
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t row = rank * nw + (threadIdx.x >> 5); row < 6 * sd.nb;
         row += (int64_t)nw * kOrthCluster) {
        const int64_t p = row / 6;
        const int c = (int)(row - 6 * p);
        const double qx = sd.q[3 * p], qy = sd.q[3 * p + 1], qz = sd.q[3 * p + 2];
        double acc = 0.0;
        for (int64_t i = sd.start[p] + lane; i < sd.start[p + 1]; i += 32) {
            const double lx = sd.x[3 * i], ly = sd.x[3 * i + 1], lz = sd.x[3 * i + 2];
            const double dx = sd.r[3 * i] - qx, dy = sd.r[3 * i + 1] - qy,
                         dz = sd.r[3 * i + 2] - qz;
            acc += c == 0 ? lx : c == 1 ? ly : c == 2 ? lz
                 : c == 3 ? dy * lz - dz * ly : c == 4 ? dz * lx - dx * lz : dx * ly - dy * lx;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) w[m3 + row] = -acc;
    }
}

// 1 / sqrt(x) in the passes' arithmetic: FP64 as rsqrt_fp64, FP32 as the
// hardware estimate refined by one Newton step
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt_fp64(x); }
__device__ __forceinline__ float rsqrt_t(float x)
{
    const float y = rsqrtf(x);
    return y * (1.5f - 0.5f * x * y * y);
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gmem) : "memory");
}

// post (optional): mapped host memory [value, count, step word]; rank 0
// writes the step word, the incremented count kept at *seq (low 32 bits)
// over the residual estimate in FP32, in one 8-byte store, so that the host
// can read the estimate without a stream synchronisation.
//
// When staged, the slices are held in T (the passes' arithmetic), so that
// FP32 passes convert each element once instead of at every use, and the
// merged coefficients of each pass are converted once as well.
template <typename T>
__global__ void __cluster_dims__(kOrthCluster, 1, 1) __launch_bounds__(kOrthClusterThreads)
    orth_cluster_kernel(double *__restrict__ V, int64_t L, int j, double *__restrict__ sm, Small S,
                        double *__restrict__ post, unsigned long long *__restrict__ seq,
                        int stage, SaddleIn sd, float *__restrict__ V32)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    // shared (slots of 8 bytes): part[2][m + 1] partial sums (pass 0; pass 1
    // with |w|^2 after pass 0 at j + 1), two spare rows, hc[m + 2] merged
    // column j of H, cs[m], sn[m] previous rotations (rank 0), red[32]
    // scalars, hT[m + 1] the summed coefficients, then (stage != 0) the
    // staged slices sV[(j + 2) x per].  The partial sums, H's column and the
    // rotations are held in T: with FP32 inner iterations (mixed precision)
    // the serial sums, the norm and the Givens update then run on the FP32
    // pipe, where a dependent operation takes a few cycles instead of the
    // ~64 of FP64 on this chip; the Hessenberg entries have the FP32
    // accuracy of the dot products they come from.
    extern __shared__ double buf[];
    const int m1 = S.m + 1;
    double *part = buf;
    T *hc = (T *)(part + 4 * m1);
    T *cs = (T *)(part + 4 * m1 + S.m + 2);
    T *sn = (T *)(part + 4 * m1 + 2 * S.m + 2);
    double *red = part + 4 * m1 + 3 * S.m + 2;
    T *hT = (T *)(red + 32);
    T *sV = (T *)(red + 32 + m1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t per = (L + kOrthCluster - 1) / kOrthCluster;
    const int64_t e0 = rank * per, e1 = e0 + per < L ? e0 + per : L;
    const int cnt = e1 > e0 ? (int)(e1 - e0) : 0;  // this CTA's slice length
    double *w = V + (int64_t)(j + 1) * L;
    // V32 (FP32 passes, staged): an FP32 copy of the basis, each vector
    // written by the step that formed it (vector 0 by step 0).  From step 1
    // on, this CTA's slices of V_0 .. V_j are copied into shared memory with
    // cp.async before the saddle rows, so that the copy overlaps them; only
    // V_{j+1} = w is staged after them.  The staged values equal T(V) either
    // way.
    const bool async_stage = stage && V32 && j >= 1;
    if (async_stage) {
        for (int x = threadIdx.x; x < (j + 1) * cnt; x += blockDim.x) {
            const int i = x / cnt, k = x - i * cnt;
            cp_async4(sV + (int64_t)i * per + k, V32 + (int64_t)i * L + e0 + k);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    if (sd.partial) {
        // w = A x from the pair kernel's partials; the cluster barrier orders
        // the body rows (written by any CTA) before every CTA's reads of w
        saddle_rows_cluster(sd, w, e0, e1, rank);
        cluster.sync();
    }
    // the Givens update's inputs from global memory, read up front into
    // red[16], red[17] (the norm uses red[0, nw))
    if (rank == 0) {
        if (threadIdx.x == 0) {
            const double gj0 = sm[S.g() + j];
            const unsigned long long q0 = post ? *seq : 0ull;
            red[16] = gj0;
            red[17] = __longlong_as_double((long long)q0);
        }
        for (int i = threadIdx.x; i < j; i += blockDim.x) {
            cs[i] = T(sm[S.cs() + i]);
            sn[i] = T(sm[S.sn() + i]);
        }
    }
    if (stage) {
        // batches of kBatch loads per thread in flight before their stores
        // (vectors i0 .. j + 1; i0 = j + 1 when V_0 .. V_j came by cp.async)
        constexpr int kBatch = 8;
        const int i0 = async_stage ? j + 1 : 0;
        const int total = (j + 2 - i0) * cnt;
        for (int x0 = threadIdx.x; x0 < total; x0 += kBatch * (int)blockDim.x) {
            double v[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int x = x0 + u * (int)blockDim.x;
                if (x < total) {
                    const int i = i0 + x / cnt, k = x % cnt;
                    v[u] = V[(int64_t)i * L + e0 + k];
                }
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int x = x0 + u * (int)blockDim.x;
                if (x < total) {
                    const int i = i0 + x / cnt, k = x % cnt;
                    sV[(int64_t)i * per + k] = T(v[u]);
                    // step 0 also leaves V_0's FP32 copy for the later steps
                    if (V32 && i == 0) V32[e0 + k] = float(v[u]);
                }
            }
        }
        if (async_stage) asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
    }
    // element e0 + k of vector i, staged (in T) or in place (FP64)
    auto ld = [&](int i, int k) -> T {
        return stage ? sV[(int64_t)i * per + k] : T(V[(int64_t)i * L + e0 + k]);
    };
    auto st_w = [&](int k, T v) {
        if (stage) sV[(int64_t)(j + 1) * per + k] = v;
        else w[e0 + k] = double(v);
    };
    // The second pass also sums |w|^2 (entry j + 1), w as the first pass
    // left it; the norm after the second pass then follows without another
    // reduction: |w2|^2 = |w1|^2 - sum_i h2_i^2, the coefficients h2 being of
    // rounding size against |w1| (the Pythagorean norm of low-synchronisation
    // CGS2), in every CTA alike from the same sums.
    T n1 = T(0);
    for (int pass = 0; pass < 2; ++pass) {
        T *pp = (T *)(part + pass * m1);
        const int top = j + pass;  // entry j + 1 of the second pass: |w|^2
        for (int i = warp; i <= top; i += nw) {
            T acc = T(0);
            for (int k = lane; k < cnt; k += 32) acc += ld(i, k) * ld(j + 1, k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) pp[i] = acc;
        }
        cluster.sync();  // every CTA's partials of this pass are written
        for (int i = threadIdx.x; i <= top; i += blockDim.x) {
            T acc = T(0);
            for (int rr = 0; rr < kOrthCluster; ++rr) acc += cluster.map_shared_rank(pp, rr)[i];
            hT[i] = acc;
            if (i <= j) hc[i] = pass == 0 ? acc : hc[i] + acc;
        }
        __syncthreads();
        if (pass == 1) n1 = hT[j + 1];
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            T acc = ld(j + 1, k);
            for (int i = 0; i <= j; ++i) acc -= ld(i, k) * hT[i];
            st_w(k, acc);
        }
        __syncthreads();  // hs, hT are rewritten by the next pass; w is final
    }
    if (threadIdx.x == 0) {
        T t = n1;
        for (int i = 0; i <= j; ++i) t -= hT[i] * hT[i];
        const T y = t > T(0) ? rsqrt_t(t) : T(0);  // 1 / |w|
        red[0] = double(t > T(0) ? t : T(0));
        red[1] = double(y);
    }
    __syncthreads();
    const double nrm2 = red[0], inv = red[1];
    if (rank == 0) {
        if (threadIdx.x == 0) {
            // Givens update of column j on the shared copy (as givens_column,
            // with the norms from reciprocal square roots), in T
            const T t = T(nrm2), yi = T(inv);
            hc[j + 1] = t * yi;
            for (int i = 0; i < j; ++i) {
                const T a = hc[i], b = hc[i + 1];
                hc[i] = cs[i] * a + sn[i] * b;
                hc[i + 1] = -sn[i] * a + cs[i] * b;
            }
            const double gj = red[16];
            const T a = hc[j], b = hc[j + 1];
            const T r2 = a * a + b * b;
            const T ir = r2 > T(0) ? rsqrt_t(r2) : T(0);
            const double c = r2 > T(0) ? double(a * ir) : 1.0;
            const double sg = r2 > T(0) ? double(b * ir) : 0.0;
            hc[j] = r2 * ir;
            hc[j + 1] = T(0);
            sm[S.cs() + j] = c;
            sm[S.sn() + j] = sg;
            sm[S.g() + j] = c * gj;
            sm[S.g() + j + 1] = -sg * gj;
            sm[S.est()] = fabs(-sg * gj);
            sm[S.nrm2()] = nrm2;
            if (post) {
                // one 8-byte store, so that no system-scope fence holds the
                // step: the count's low 32 bits over the estimate in FP32
                // (the precision of the inner stopping test it serves)
                const unsigned long long q = (unsigned long long)__double_as_longlong(red[17]) + 1;
                *seq = q;
                const float e32 = (float)fabs(-sg * gj);
                *(volatile unsigned long long *)(post + 2) = (q << 32) | __float_as_uint(e32);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) sm[S.H(i, j)] = double(hc[i]);
    }
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
        const double v = double(ld(j + 1, k)) * inv;
        w[e0 + k] = v;
        if (V32 && stage) V32[(int64_t)(j + 1) * L + e0 + k] = float(v);
    }
    cluster.sync();  // no CTA exits while another still reads its partials; w is final
}

// body of every blob, for the small-system steps
__global__ void body_map_kernel(const int64_t *__restrict__ start, int64_t nb, int64_t n,
                                int *__restrict__ body)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        body[i] = (int)body_of(start, nb, i);
}


size_t orth_cluster_smem(int m) { return sizeof(double) * (8 * (size_t)m + 39); }

// Whether step j stages its slices, and its dynamic shared memory.
bool orth_cluster_stage(int64_t L, int j)
{
    return (int64_t)(j + 2) * ((L + kOrthCluster - 1) / kOrthCluster) <= kOrthStageDoubles;
}
size_t orth_cluster_step_smem(int m, int64_t L, int j)
{
    return orth_cluster_smem(m) +
           (orth_cluster_stage(L, j)
                ? sizeof(double) * (size_t)(j + 2) * (size_t)((L + kOrthCluster - 1) / kOrthCluster)
                : 0);
}

// h[i] += y[i] for i <= j: the second CGS pass's coefficients (held in y)
__global__ void merge_passes_kernel(double *__restrict__ sm, Small L, int j)
{
    for (int i = threadIdx.x; i <= j; i += blockDim.x) sm[L.h() + i] += sm[L.y() + i];
}

// Back substitution R y = g for the leading k x k triangle.
// 1/d in FP64: the FP32 reciprocal refined by two FP64 Newton steps
// y <- y (2 - d y); arguments outside the FP32 range take the division.
__device__ __forceinline__ double rcp_fp64(double d)
{
    const double ad = fabs(d);
    if (!(ad > 1e-30 && ad < 1e30)) return 1.0 / d;
    double y = (double)(1.0f / (float)d);
    y = y * (2.0 - d * y);
    return y * (2.0 - d * y);
}

// y = R^-1 g for the k x k upper triangle R of H (the least-squares problem
// of the restart cycle).  For k <= 32 one warp runs it: lane i holds row i,
// all reciprocals of the diagonal are formed at once, and the back
// substitution is column-oriented (y_j, once known, is subtracted from every
// earlier row at once): one shuffle and one FMA per step instead of a
// division and a dot product.  Larger k take the serial loop on one thread.
__global__ void solve_triangle_kernel(double *__restrict__ sm, Small L, int k)
{
    const int lane = threadIdx.x & 31;
    if (k <= 32) {
        if (threadIdx.x >= 32) return;
        // row `lane` of R in registers first: the loads are all in flight at
        // once instead of one per step of the chain
        double h[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) h[j] = lane < j && j < k ? sm[L.H(lane, j)] : 0.0;
        const double d = lane < k ? sm[L.H(lane, lane)] : 1.0;
        const double rinv = d != 0.0 ? rcp_fp64(d) : 0.0;
        double acc = lane < k ? sm[L.g() + lane] : 0.0;
#pragma unroll
        for (int j = 31; j >= 0; --j) {
            if (j < k) {
                const double yj = __shfl_sync(0xffffffffu, acc * rinv, j);
                if (lane == j) acc = yj;
                else if (lane < j) acc -= h[j] * yj;
            }
        }
        if (lane < k) sm[L.y() + lane] = acc;
        return;
    }
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double acc = sm[L.g() + i];
        for (int j = i + 1; j < k; ++j) acc -= sm[L.H(i, j)] * sm[L.y() + j];
        const double d = sm[L.H(i, i)];
        sm[L.y() + i] = d != 0.0 ? acc / d : 0.0;
    }
}

// b = [slip or 0 ; -(F, T) interleaved per body]
__global__ void build_rhs_kernel(int64_t n, int64_t nb, const double *__restrict__ slip,
                                 const double *__restrict__ F, const double *__restrict__ T,
                                 double *__restrict__ b)
{
    const int64_t L = 3 * n + 6 * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < 3 * n) {
            b[e] = slip ? slip[e] : 0.0;
        } else {
            const int64_t k = e - 3 * n, p = k / 6, c = k % 6;
            b[e] = c < 3 ? -F[3 * p + c] : -T[3 * p + c - 3];
        }
    }
}

__global__ void unpack_solution_kernel(int64_t n, int64_t nb, const double *__restrict__ x,
                                       double *__restrict__ U, double *__restrict__ Om,
                                       double *__restrict__ lam)
{
    const int64_t L = 3 * n + 6 * nb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < 3 * n) {
            lam[e] = x[e];
        } else {
            const int64_t k = e - 3 * n, p = k / 6, c = k % 6;
            if (c < 3) U[3 * p + c] = x[e];
            else Om[3 * p + c - 3] = x[e];
        }
    }
}

// b = K [U; Omega] + slip on the blobs (resistance right-hand side)
__global__ void build_rhs_resist_kernel(int64_t nb, int64_t n, const double *__restrict__ r,
                                        const double *__restrict__ q,
                                        const int64_t *__restrict__ start,
                                        const double *__restrict__ U,
                                        const double *__restrict__ Om,
                                        const double *__restrict__ slip, double *__restrict__ b)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = nb;  // body of blob i: start[lo] <= i < start[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (start[mid] <= i) lo = mid;
            else hi = mid;
        }
        const double dx = r[3 * i] - q[3 * lo], dy = r[3 * i + 1] - q[3 * lo + 1],
                     dz = r[3 * i + 2] - q[3 * lo + 2];
        const double *u = U + 3 * lo, *w = Om + 3 * lo;
        const double v[3] = {u[0] + (w[1] * dz - w[2] * dy), u[1] + (w[2] * dx - w[0] * dz),
                             u[2] + (w[0] * dy - w[1] * dx)};
#pragma unroll
        for (int c = 0; c < 3; ++c) b[3 * i + c] = v[c] + (slip ? slip[3 * i + c] : 0.0);
    }
}

// y_i += shift_i x_i on the blob part (permeable bodies: Appendix C adds
// kappa_p / (eta dV_i) to the diagonal of M)
__global__ void add_shift_kernel(double *__restrict__ y, const double *__restrict__ x,
                                 const double *__restrict__ shift, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] += shift[e / 3] * x[e];
}

// F, T from the packed n_b x 6 K^T lambda
__global__ void split_ft_kernel(int64_t nb, const double *__restrict__ FT, double *__restrict__ F,
                                double *__restrict__ T)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 6 * nb;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / 6, c = e % 6;
        if (c < 3) F[3 * p + c] = FT[e];
        else T[3 * p + c - 3] = FT[e];
    }
}

struct Solver {
    mb_context *ctx;
    bool resist = false;  // A = M alone (resistance problem), L = 3N
    bool pc_f32 = false;  // apply the preconditioner from its FP32 copy (FP32 inner iterations)
    const double *shift = nullptr;  // per-blob diagonal addition to M, or null
    cudaStream_t s;
    int64_t n, nb, L;
    const double *r, *q;
    const int64_t *start;
    double a, eta;
    int wall;
    int m;
    Small sl;
    double *V, *Z, *b, *x, *w, *t, *sm, *partial;
    double *hsm;  // pinned host mirror (2 doubles)

    // y = A x with the pair kernel in precision `prec`.  When the pair
    // kernel leaves chunk partials, their reduction and both kinematic rows
    // run as one launch (saddle_rows_kernel) instead of three.
    // keep (optional): when the rows are fused and the pair kernel left
    // partials, launch nothing more and describe them there (the caller's
    // next kernel forms y, see saddle_rows_cluster).
    mb_status apply_A(const double *xin, double *y, mb_precision prec, SaddleIn *keep = nullptr)
    {
        MatvecPartials mp;
        const bool fuse = !shift && !resist && nb >= 1 && nb <= kSaddleRowsMaxBodies;
        MB_TRY(matvec_packed(ctx, r, xin, n, a, eta, wall, prec, y, s, fuse ? &mp : nullptr));
        if (mp.S > 0 && keep) {
            keep->partial = mp.partial; keep->S = mp.S; keep->scale = mp.scale;
            keep->n = n; keep->nb = nb; keep->r = r; keep->q = q; keep->start = start;
            keep->x = xin;
            return MB_OK;
        }
        if (mp.S > 0) {
            launch_saddle_rows(mp, n, nb, r, q, start, xin, y, s);
            MB_CUDA_TRY(ctx, cudaGetLastError());
            return MB_OK;
        }
        if (shift) {
            add_shift_kernel<<<vec_grid(3 * n), 256, 0, s>>>(y, xin, shift, n);
            count_launch();
        }
        if (resist) return MB_OK;
        launch_K_apply(nb, n, r, q, start, xin + 3 * n, y, -1.0, 1.0, s);
        launch_KT_apply(nb, r, q, start, xin, y + 3 * n, -1.0, s);
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }

    // y = A x from the running sum y_M += M dx_lambda (pair kernel in `prec`)
    mb_status apply_A_incremental(const double *xin, const double *dx, double *ym, double *y,
                                  mb_precision prec)
    {
        MB_TRY(matvec_packed(ctx, r, dx, n, a, eta, wall, prec, y, s));
        if (shift) {
            add_shift_kernel<<<vec_grid(3 * n), 256, 0, s>>>(y, dx, shift, n);
            count_launch();
        }
        accumulate_kernel<<<vec_grid(3 * n), 256, 0, s>>>(y, ym, 3 * n);
        count_launch();
        if (resist) return MB_OK;
        launch_K_apply(nb, n, r, q, start, xin + 3 * n, y, -1.0, 1.0, s);
        launch_KT_apply(nb, r, q, start, xin, y + 3 * n, -1.0, s);
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }

    // z = P^-1 v (the indefinite blocks, or the blob blocks alone)
    void precond(const double *v, double *z, cudaStream_t cs)
    {
        if (resist) precond_apply_blobs(ctx, v, z, cs);
        else precond_apply_packed(ctx, v, z, cs, pc_f32);
    }

    // out[0..nk) = V[0..nk) . w  (accumulate: out += ...)
    void dots(const double *Vb, int nk, const double *wv, double *out, int accumulate)
    {
        const int nblk = (int)std::min<int64_t>(kRedBlocks, ceil_div(L, kRedThreads));
        multidot_kernel<<<dim3(nblk, nk), kRedThreads, 0, s>>>(Vb, L, nk, wv, L, partial);
        count_launch();
        finish_dots_kernel<<<nk, 32, 0, s>>>(partial, nblk, nk, out, accumulate);
        count_launch();
    }

    // The estimate posted by the kernel just launched: poll the mapped count
    // for up to 2 ms, then fall back to a stream synchronisation (long steps,
    // or no mapped memory), which also resynchronises the count.  A cycle
    // start posts [value, count] in FP64 behind a fence; an Arnoldi step
    // (`step`) posts one word, the count's low 32 bits over an FP32 estimate.
    mb_status read_posted_est(double *est, bool step = false)
    {
        if (!ctx->host_post) return read_est(est);
        const unsigned long long want = ++ctx->post_seq;
        volatile unsigned long long *cnt = (volatile unsigned long long *)(ctx->host_post + 1);
        volatile unsigned long long *word = (volatile unsigned long long *)(ctx->host_post + 2);
        const auto t0 = std::chrono::steady_clock::now();
        for (long it = 0;; ++it) {
            if (step) {
                const unsigned long long wv = *word;
                if ((int32_t)((uint32_t)(wv >> 32) - (uint32_t)want) >= 0) {
                    const uint32_t bits = (uint32_t)wv;
                    float e;
                    std::memcpy(&e, &bits, sizeof e);
                    *est = (double)e;
                    return MB_OK;
                }
            } else if (*cnt >= want) {
                std::atomic_thread_fence(std::memory_order_acquire);
                *est = *(volatile double *)ctx->host_post;
                return MB_OK;
            }
            if ((it & 255) == 255) {
                const double el = std::chrono::duration<double>(
                                      std::chrono::steady_clock::now() - t0).count();
                if (ctx->wait_limit_s > 0.0 && el > ctx->wait_limit_s)
                    return set_err(ctx, MB_ETIMEOUT,
                                   "Krylov step: no estimate posted after %.3g s (wait limit); "
                                   "the enqueued work still runs, synchronise the stream before "
                                   "the next call", ctx->wait_limit_s);
                if (el > 2e-3) break;
            }
        }
        MB_TRY(read_est(est));
        ctx->post_seq = posted_count(ctx->host_post);  // the stream is idle: every posting has arrived
        return MB_OK;
    }

    mb_status read_est(double *est)
    {
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(hsm, sm + sl.est(), sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
        MB_TRY(wait_stream(ctx, s, "Krylov step"));
        *est = hsm[0];
        return MB_OK;
    }
};

// The cache entry for a step signature: the matching one, else a free slot,
// else the least recently used entry (its graph destroyed).
IterGraph &graph_entry(mb_context *ctx, const IterSig &sig)
{
    auto &v = ctx->iter_graphs;
    IterGraph *hit = nullptr;
    for (auto &g : v)
        if (g.sig == sig) { hit = &g; break; }
    if (!hit) {
        if (v.size() < kMaxIterGraphs) {
            v.emplace_back();
            hit = &v.back();
        } else {
            hit = &v[0];
            for (auto &g : v)
                if (g.last_use < hit->last_use) hit = &g;
            if (hit->exec) cudaGraphExecDestroy(hit->exec);
            *hit = IterGraph{};
        }
    }
    hit->last_use = ++ctx->graph_clock;
    return *hit;
}

// Run one Arnoldi step through its cached graph: replay it when the
// signature matches, capture it when this signature was met once before,
// otherwise only record the signature (the caller then runs the step
// directly).  *ran tells whether the step was launched here.  A capture
// that fails for any reason is dropped and the step runs directly.
template <typename Step>
mb_status run_step_graph(mb_context *ctx, IterGraph &g, const IterSig &sig, Step &step,
                         cudaStream_t s, bool *ran)
{
    *ran = false;
    if (g.exec && g.sig == sig) {
        MB_CUDA_TRY(ctx, cudaGraphLaunch(g.exec, s));
        count_launch(g.launches);
        *ran = true;
        return MB_OK;
    }
    if (g.exec) {
        cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    if (!(g.seen && g.sig == sig)) {
        g.seen = true;
        g.sig = sig;
        return MB_OK;
    }
    // capture on the context's own stream (capture is not allowed on the
    // legacy default stream); nothing executes until the launch on s
    if (!ctx->cap_stream &&
        cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        ctx->cap_stream = nullptr;
        cudaGetLastError();
        return MB_OK;
    }
    const long long l0 = g_launches.load();
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return MB_OK;
    }
    const std::string saved_err = ctx->err;
    const mb_status st = step(ctx->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    const long long captured = g_launches.load() - l0;
    count_launch(-captured);  // nothing ran yet
    if (st != MB_OK || e != cudaSuccess || !graph ||
        cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        g.exec = nullptr;
        g.seen = false;
        cudaGetLastError();
        ctx->err = saved_err;
        return MB_OK;
    }
    cudaGraphDestroy(graph);
    g.launches = captured;
    MB_CUDA_TRY(ctx, cudaGraphLaunch(g.exec, s));
    count_launch(g.launches);
    *ran = true;
    return MB_OK;
}

}  // namespace

// Mobility problem (resist = 0): inputs in_a, in_b = F, T; outputs out_a,
// out_b = U, Omega.  Resistance problem (resist = 1): inputs U, Omega;
// outputs F, T.  lambda is the blob-force output of both.
static mb_status solve_rigid(mb_context *ctx, int resist, int64_t nb, int64_t n, const double *q,
                             const double *theta, const int64_t *blob_start, const double *rho,
                             const double *in_a, const double *in_b, const double *slip,
                             const mb_params *p, double *out_a, double *out_b, double *lambda,
                             mb_info *info, cudaStream_t s, const double *shift)
{
    using clk = std::chrono::steady_clock;
    const auto t0 = clk::now();
    const int m = std::max(1, std::min(p->restart, 500));
    const int64_t L = resist ? 3 * n : 3 * n + 6 * nb;
    Small sl{m};

    MB_TRY(ensure(ctx, ctx->sol_r, sizeof(double) * 3 * n, "blob positions"));
    MB_TRY(ensure(ctx, ctx->sol_V, sizeof(double) * L * (m + 1), "Krylov basis V"));
    MB_TRY(ensure(ctx, ctx->sol_Z, sizeof(double) * L * m, "Krylov basis Z"));
    MB_TRY(ensure(ctx, ctx->sol_b, sizeof(double) * L, "rhs"));
    MB_TRY(ensure(ctx, ctx->sol_x, sizeof(double) * L, "iterate"));
    MB_TRY(ensure(ctx, ctx->sol_w, sizeof(double) * L, "work vector"));
    MB_TRY(ensure(ctx, ctx->sol_t, sizeof(double) * std::max<int64_t>(L, 6 * nb), "work vector"));
    const bool mixed = p->prec == MB_MIXED_REFINE;
    if (mixed) {
        MB_TRY(ensure(ctx, ctx->sol_dx, sizeof(double) * L, "cycle correction"));
        MB_TRY(ensure(ctx, ctx->sol_ym, sizeof(double) * 3 * n, "running M lambda"));
    }
    MB_TRY(ensure(ctx, ctx->sol_small, sizeof(double) * (sl.total() + (m + 1) * kRedBlocks),
                  "Krylov scalars"));
    if (!ctx->host_small) MB_CUDA_TRY(ctx, cudaMallocHost(&ctx->host_small, 64));
    if (!ctx->host_post) {
        // mapped memory for posted estimates; without it the estimates are
        // read after a stream synchronisation
        void *hp = nullptr, *dp = nullptr;
        unsigned long long *sq = nullptr;
        if (cudaHostAlloc(&hp, 64, cudaHostAllocMapped) == cudaSuccess &&
            cudaHostGetDevicePointer(&dp, hp, 0) == cudaSuccess &&
            cudaMalloc(&sq, sizeof(unsigned long long)) == cudaSuccess &&
            cudaMemset(sq, 0, sizeof(unsigned long long)) == cudaSuccess) {
            std::memset(hp, 0, 64);
            ctx->host_post = (double *)hp;
            ctx->host_post_dev = (double *)dp;
            ctx->post_seq_dev = sq;
            ctx->post_seq = 0;
        } else {
            if (hp) cudaFreeHost(hp);
            if (sq) cudaFree(sq);
            cudaGetLastError();
        }
    }

    double *r = (double *)ctx->sol_r.ptr;
    MB_TRY(blob_positions(ctx, nb, n, q, theta, blob_start, rho, r, s));
    if (p->precond == MB_PRECOND_FREE_SHARED)
        MB_TRY(precond_setup_shared(ctx, nb, n, theta, blob_start, rho, p->a, p->eta, s, !resist));
    else
        MB_TRY(precond_setup(ctx, nb, n, r, q, blob_start, p->a, p->eta, p->wall, s, !resist,
                             shift));
    if (p->prec != MB_FP64) MB_TRY(matvec_pack_positions(ctx, r, n, s));
    MB_TRY(wait_stream(ctx, s, "solver setup"));
    const auto t1 = clk::now();
    // the stream is idle, so every posting of earlier calls has arrived (an
    // earlier call that ran out of its wait limit may have left some behind)
    if (ctx->host_post) ctx->post_seq = posted_count(ctx->host_post);

    Solver S;
    S.resist = resist != 0;
    S.shift = shift;
    S.ctx = ctx; S.s = s; S.n = n; S.nb = nb; S.L = L; S.r = r; S.q = q;
    S.start = (const int64_t *)ctx->blob_start_copy.ptr;
    S.a = p->a; S.eta = p->eta; S.wall = p->wall; S.m = m; S.sl = sl;
    S.V = (double *)ctx->sol_V.ptr; S.Z = (double *)ctx->sol_Z.ptr;
    S.b = (double *)ctx->sol_b.ptr; S.x = (double *)ctx->sol_x.ptr;
    S.w = (double *)ctx->sol_w.ptr; S.t = (double *)ctx->sol_t.ptr;
    S.sm = (double *)ctx->sol_small.ptr; S.partial = S.sm + sl.total();
    S.hsm = (double *)ctx->host_small;

    const mb_precision inner = inner_precision(p->prec);
    const mb_precision outer = outer_precision(p->prec);
    const int vg = vec_grid(L);
    // FP32 inner iterations apply the explicit blocks from an FP32 copy (the
    // flexible GMRES keeps the z_j it was given)
    if (inner == MB_FP32_KAHAN && !resist && p->precond != MB_PRECOND_FREE_SHARED) {
        MB_TRY(precond_make_f32(ctx, s));
        S.pc_f32 = ctx->pc_f32_ready;
    }
    // small systems with FP32 passes: the basis' FP32 copy (see orth_cluster_kernel)
    float *V32 = nullptr;
    if (L <= kOrthSmallMax && inner == MB_FP32_KAHAN) {
        MB_TRY(ensure(ctx, ctx->sol_V32, sizeof(float) * (size_t)L * (m + 1), "FP32 Krylov basis"));
        V32 = (float *)ctx->sol_V32.ptr;
    }
    // small systems: the body of every blob, for the saddle rows formed in the
    // orthogonalisation
    const int *body_map = nullptr;
    if (L <= kOrthSmallMax && !resist) {
        MB_TRY(ensure(ctx, ctx->sol_body, sizeof(int) * (size_t)n, "blob bodies"));
        body_map_kernel<<<vec_grid(n), 256, 0, s>>>(S.start, nb, n, (int *)ctx->sol_body.ptr);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
        body_map = (const int *)ctx->sol_body.ptr;
    }
    if (L <= kOrthSmallMax) {
        // a step that stages its slices may need more than 48 KB of shared memory
        const int smax = (int)(orth_cluster_smem(m) + sizeof(double) * kOrthStageDoubles);
        MB_CUDA_TRY(ctx, cudaFuncSetAttribute(orth_cluster_kernel<float>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        MB_CUDA_TRY(ctx, cudaFuncSetAttribute(orth_cluster_kernel<double>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
    }

    if (resist)
        build_rhs_resist_kernel<<<vec_grid(n), 256, 0, s>>>(nb, n, r, q, S.start, in_a, in_b, slip,
                                                            S.b);
    else
        build_rhs_kernel<<<vg, 256, 0, s>>>(n, nb, slip, in_a, in_b, S.b);
    count_launch();
    MB_CUDA_TRY(ctx, cudaMemsetAsync(S.x, 0, sizeof(double) * L, s));
    double *dx = mixed ? (double *)ctx->sol_dx.ptr : nullptr;
    double *ym = mixed ? (double *)ctx->sol_ym.ptr : nullptr;
    if (mixed) MB_CUDA_TRY(ctx, cudaMemsetAsync(ym, 0, sizeof(double) * 3 * n, s));
    S.dots(S.b, 1, S.b, S.sm + sl.nrm2(), 0);
    MB_CUDA_TRY(ctx, cudaGetLastError());
    double bnorm2 = 0.0;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(S.hsm, S.sm + sl.nrm2(), sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
    MB_TRY(wait_stream(ctx, s, "right-hand side norm"));
    bnorm2 = S.hsm[0];
    const double bnorm = std::sqrt(bnorm2);

    int iters = 0, restarts = 0, converged = 0;
    double rel = 0.0;
    if (!(bnorm > 0.0)) {
        converged = 1;  // x = 0 solves b = 0
    } else {
        for (;;) {
            // true residual w = b - A x
            if (iters == 0) {
                MB_CUDA_TRY(ctx, cudaMemcpyAsync(S.w, S.b, sizeof(double) * L,
                                                 cudaMemcpyDeviceToDevice, s));
            } else {
                if (mixed) {
                    // rel still holds the residual this cycle started from
                    const bool fine = rel <= kFineRel * p->tol;
                    MB_TRY(S.apply_A_incremental(S.x, dx, ym, S.t, fine ? inner : outer));
                } else {
                    MB_TRY(S.apply_A(S.x, S.t, outer));
                }
                sub_kernel<<<vg, 256, 0, s>>>(S.b, S.t, S.w, L);
                count_launch();
            }
            S.dots(S.w, 1, S.w, S.sm + sl.nrm2(), 0);
            cycle_start_kernel<<<1, 1, 0, s>>>(S.sm, sl, ctx->host_post_dev, ctx->post_seq_dev);
            count_launch();
            double beta = 0.0;
            MB_TRY(S.read_posted_est(&beta));
            rel = beta / bnorm;
            if (!std::isfinite(rel))
                return set_err(ctx, MB_ESINGULAR, "non-finite residual (check blob heights)");
            if (rel <= p->tol) {
                converged = 1;
                break;
            }
            if (iters >= p->maxit) break;
            // inner tolerance: the final target, or (mixed) a 1e-5 reduction per cycle
            double inner_abs = 0.5 * p->tol * bnorm;
            if (p->prec == MB_MIXED_REFINE) inner_abs = std::max(inner_abs, 1e-5 * beta);
            scale_kernel<<<vg, 256, 0, s>>>(S.w, S.V, L, S.sm + sl.nrm2(), 1);
            count_launch();
            int k = 0;
            for (int j = 0; j < m && iters < p->maxit; ++j) {
                double *vj = S.V + (int64_t)j * L;
                double *zj = S.Z + (int64_t)j * L;
                double *vn = S.V + (int64_t)(j + 1) * L;
                ++iters;
                k = j + 1;
                if ((int64_t)(j + 1) * L <= kOrthSmallMax) {
                    // small system: preconditioner, matvec and the one-CTA
                    // orthogonalisation, replayed as a CUDA graph once captured
                    auto step = [&](cudaStream_t cs) -> mb_status {
                        S.s = cs;
                        S.precond(vj, zj, cs);
                        SaddleIn sd;
                        const mb_status st = S.apply_A(zj, vn, inner, &sd);
                        S.s = s;
                        if (st != MB_OK) return st;
                        sd.body = body_map;
                        const size_t osm = orth_cluster_step_smem(m, L, j);
                        const int stage = orth_cluster_stage(L, j) ? 1 : 0;
                        if (inner == MB_FP32_KAHAN)
                            orth_cluster_kernel<float><<<kOrthCluster, kOrthClusterThreads, osm, cs>>>(
                                S.V, L, j, S.sm, sl, ctx->host_post_dev, ctx->post_seq_dev, stage, sd,
                                V32);
                        else
                            orth_cluster_kernel<double><<<kOrthCluster, kOrthClusterThreads, osm, cs>>>(
                                S.V, L, j, S.sm, sl, ctx->host_post_dev, ctx->post_seq_dev, stage, sd,
                                nullptr);
                        count_launch();
                        MB_CUDA_TRY(ctx, cudaGetLastError());
                        return MB_OK;
                    };
                    bool ran = false;
                    if (!ctx->profiling) {
                        IterSig sig;
                        sig.gen = ctx->alloc_gen; sig.j = j; sig.m = m; sig.inner = (int)inner;
                        sig.wall = p->wall; sig.variant = ctx->pair_variant;
                        sig.pc_max_np = ctx->pc_max_np; sig.pc_kind = ctx->pc_kind;
                        sig.pc_factored = ctx->pc_factored;
                        sig.mode = resist;
                        sig.shift = shift;
                        sig.n = n; sig.nb = nb; sig.L = L;
                        sig.pc_nb = ctx->pc_nb; sig.a = p->a; sig.eta = p->eta; sig.q = q;
                        sig.V = S.V; sig.Z = S.Z; sig.sm = S.sm;
                        MB_TRY(run_step_graph(ctx, graph_entry(ctx, sig), sig, step, s, &ran));
                    }
                    if (!ran) MB_TRY(step(s));
                    double est = 0.0;
                    MB_TRY(S.read_posted_est(&est, true));
                    if (!(est > inner_abs)) break;
                    continue;
                }
                S.precond(vj, zj, s);
                MB_TRY(S.apply_A(zj, vn, inner));
                // CGS2
                S.dots(S.V, j + 1, vn, S.sm + sl.h(), 0);
                subtract_span_kernel<<<vg, 256, 0, s>>>(S.V, L, j + 1, S.sm + sl.h(), vn, L);
                count_launch();
                S.dots(S.V, j + 1, vn, S.sm + sl.y(), 0);
                subtract_span_kernel<<<vg, 256, 0, s>>>(S.V, L, j + 1, S.sm + sl.y(), vn, L);
                count_launch();
                S.dots(vn, 1, vn, S.sm + sl.nrm2(), 0);
                // merge the two Gram-Schmidt passes into column j, then rotate
                merge_passes_kernel<<<1, 32, 0, s>>>(S.sm, sl, j);
                count_launch();
                MB_CUDA_TRY(ctx, cudaGetLastError());
                givens_kernel<<<1, 1, 0, s>>>(S.sm, sl, j);
                count_launch();
                scale_kernel<<<vg, 256, 0, s>>>(vn, vn, L, S.sm + sl.nrm2(), 1);
                count_launch();
                double est = 0.0;
                MB_TRY(S.read_est(&est));
                if (!(est > inner_abs)) break;
            }
            solve_triangle_kernel<<<1, 32, 0, s>>>(S.sm, sl, k);
            count_launch();
            if (mixed)
                update_span_kernel<<<vg, 256, 0, s>>>(S.Z, L, k, S.sm + sl.y(), S.x, dx, L);
            else
                add_span_kernel<<<vg, 256, 0, s>>>(S.Z, L, k, S.sm + sl.y(), S.x, L);
            count_launch();
            MB_CUDA_TRY(ctx, cudaGetLastError());
            ++restarts;
        }
    }
    if (resist) {
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(lambda, S.x, sizeof(double) * 3 * n,
                                         cudaMemcpyDeviceToDevice, s));
        launch_KT_apply(nb, r, q, S.start, S.x, S.t, 1.0, s);
        split_ft_kernel<<<vec_grid(6 * nb), 256, 0, s>>>(nb, S.t, out_a, out_b);
    } else {
        unpack_solution_kernel<<<vg, 256, 0, s>>>(n, nb, S.x, out_a, out_b, lambda);
    }
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    MB_TRY(wait_stream(ctx, s, "solution"));
    const auto t2 = clk::now();
    if (info) {
        info->iters = iters;
        info->restarts = restarts;
        info->converged = converged;
        info->rel_residual = rel;
        info->setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        info->solve_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
    }
    if (!converged)
        return set_err(ctx, MB_ENOTCONVERGED, "GMRES reached maxit=%d with relative residual %.3e",
                       p->maxit, rel);
    return MB_OK;
}

mb_status solve_mobility(mb_context *ctx, int64_t nb, int64_t n, const double *q,
                         const double *theta, const int64_t *blob_start, const double *rho,
                         const double *F, const double *T, const double *slip,
                         const mb_params *p, double *U, double *Omega, double *lambda,
                         mb_info *info, cudaStream_t s, const double *shift)
{
    return solve_rigid(ctx, 0, nb, n, q, theta, blob_start, rho, F, T, slip, p, U, Omega, lambda,
                       info, s, shift);
}

mb_status solve_resistance(mb_context *ctx, int64_t nb, int64_t n, const double *q,
                           const double *theta, const int64_t *blob_start, const double *rho,
                           const double *U, const double *Omega, const double *slip,
                           const mb_params *p, double *F, double *T, double *lambda,
                           mb_info *info, cudaStream_t s)
{
    return solve_rigid(ctx, 1, nb, n, q, theta, blob_start, rho, U, Omega, slip, p, F, T, lambda,
                       info, s, nullptr);
}

}  // namespace mb
