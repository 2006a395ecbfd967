// Continuous-batching engine for mobility solves (mb_server_*, mb_solve_batch).
//
// A server owns one device arena sized at creation: blob, body and
// preconditioner ranges plus Krylov vectors laid out as
//     x = [lambda of every blob slot (3 N_cap) | (U, Omega) of every body slot (6 B_cap)].
// A request is admitted when contiguous blob, body and preconditioner ranges
// fit (first fit), i.e. by its HBM footprint.  The queue is scanned in
// arrival order and every request that fits is admitted, so a small request
// does not wait behind a large one that does not fit yet; a queued request
// that later ones have overtaken max_bypass times stops the scan until it is
// admitted itself (aging), which bounds its wait.  Its positions, right-hand side,
// factorised preconditioner blocks and Krylov state then stay on the device
// until it completes.  Each scheduling tick
//   1. retires finished requests (results scattered to the caller's arrays,
//      ranges freed) and admits queued ones (blob build, preconditioner setup
//      of Section 2.2.2, right-hand side);
//   2. computes the true residual b - A x for every request starting a
//      restart cycle (one batched matvec in the outer precision; in mixed
//      precision a batched product of the last cycle's correction, added to
//      each request's FP64 running sum of M lambda, in FP32 once the
//      correction is small enough for its error to stay under a tenth of the
//      tolerance, as in the single-problem solver);
//   3. runs one Arnoldi step of right-preconditioned flexible GMRES for every
//      active request, whatever its step index: one batched preconditioner
//      apply, one batched pair-kernel launch over all requests' (target
//      block, source chunk) items, segmented CGS2 reductions and Givens
//      rotations per request.
// Requests therefore join and leave between iterations while others are in
// flight, and all of them share the same kernel launches.  mb_solve_batch is
// this engine with every problem submitted at once and run to completion.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <new>
#include <string>
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
constexpr int64_t kSeg = 4096;   // elements per vector chunk item
constexpr int kRT = 256;         // threads of reduction kernels

using clk = std::chrono::steady_clock;

// ------------------------------------------------------------------ device records
struct Seg {          // chunk [start, end) of the global vector owned by `slot`
    int64_t start, end;
    int slot, pad;
};

struct Work {         // pair-kernel work of one request in one launch
    const float4 *hi, *lo;
    const double *r, *f;
    double *y, *part;
    int64_t n, chunk, item_off;
    int n_tblocks, S, slot, tri_lo;  // tri_lo: first block-pair item (symmetric, split matvecs)
};

struct RSeg {         // chunk of a work entry's local rows for the partial reduction
    int64_t start, end;
    int work, pad;
};

struct SlotIn {       // inputs of a request being admitted
    const double *q, *theta, *rho, *F, *T, *slip;
    const int64_t *blob_start;
    int64_t n, nb, blob_off, body_off, start_off;
};

struct SlotOut {      // outputs of a request being retired
    double *U, *Omega, *lambda;
    int64_t n, nb, blob_off, body_off;
};

// Per-slot Krylov scalars (doubles), stride total():
//   H[(m+1) x m] column-major, cs[m], sn[m], g[m+1], y[m], h[m+1], nrm2, est,
//   bnorm, inner, rel
struct SL {
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

struct SlotState {    // per-slot device integers
    int *act;         // doing an Arnoldi step this tick
    int *live;        // admitted and not finished
    int *conv;        // converged
    int *j;           // Arnoldi step index within the cycle
    int *iters;       // total Arnoldi steps
    int *restarts;    // completed cycles
    int *park;        // cycle ended this tick
    int *bad;         // set at admission: 1 malformed descriptor, 2 singular block
    int *fine;        // mixed: the running cycle's correction may be multiplied in FP32
};

constexpr int kSlotInts = 9;  // int arrays in SlotState
// mixed precision: FP32 increments once a cycle starts below kFineRel * tol * |b|
constexpr double kFineRel = 1e4;

__device__ __forceinline__ int find_owner(const int64_t *__restrict__ off, int n, int64_t item)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ admission
__global__ void admit_kernel(const SlotIn *__restrict__ in, int nin, const int *__restrict__ slot_of,
                             double *rho, double *slip, double *q, double *theta, double *F,
                             double *T, int64_t *bstart, int64_t *body_b0, int64_t *body_b1,
                             int *blob_slot, int *body_slot, int64_t *blob_body, int *bad)
{
    for (int k = blockIdx.x; k < nin; k += gridDim.x) {
        const SlotIn d = in[k];
        const int s = slot_of[k];
        if (threadIdx.x == 0) bad[s] = (d.blob_start[0] != 0 || d.blob_start[d.nb] != d.n) ? 1 : 0;
        for (int64_t e = threadIdx.x; e < 3 * d.n; e += blockDim.x) {
            rho[3 * d.blob_off + e] = d.rho[e];
            slip[3 * d.blob_off + e] = d.slip ? d.slip[e] : 0.0;
        }
        for (int64_t e = threadIdx.x; e < d.n; e += blockDim.x) blob_slot[d.blob_off + e] = s;
        for (int64_t e = threadIdx.x; e <= d.nb; e += blockDim.x) {
            int64_t b = d.blob_start[e];
            b = b < 0 ? 0 : (b > d.n ? d.n : b);  // keep a malformed descriptor in range
            bstart[d.start_off + e] = d.blob_off + b;
        }
        for (int64_t e = threadIdx.x; e < d.nb; e += blockDim.x) {
            const int64_t b = d.body_off + e;
            for (int c = 0; c < 3; ++c) {
                q[3 * b + c] = d.q[3 * e + c];
                F[3 * b + c] = d.F[3 * e + c];
                T[3 * b + c] = d.T[3 * e + c];
            }
            for (int c = 0; c < 4; ++c) theta[4 * b + c] = d.theta[4 * e + c];
            body_slot[b] = s;
        }
        __syncthreads();
        for (int64_t e = threadIdx.x; e < d.nb; e += blockDim.x) {
            const int64_t b = d.body_off + e;
            const int64_t b0 = bstart[d.start_off + e], b1 = bstart[d.start_off + e + 1];
            body_b0[b] = b0;
            body_b1[b] = b1 > b0 ? b1 : b0;
            for (int64_t i = b0; i < b1; ++i) blob_body[i] = b;
        }
    }
}

// release: mark the freed ranges as holes
__global__ void release_kernel(const SlotOut *__restrict__ out, int nout, int *blob_slot,
                               int *body_slot, int64_t *blob_body)
{
    for (int k = blockIdx.x; k < nout; k += gridDim.x) {
        const SlotOut d = out[k];
        for (int64_t e = threadIdx.x; e < d.n; e += blockDim.x) {
            blob_slot[d.blob_off + e] = -1;
            blob_body[d.blob_off + e] = -1;
        }
        for (int64_t e = threadIdx.x; e < d.nb; e += blockDim.x) body_slot[d.body_off + e] = -1;
    }
}

__global__ void scatter_kernel(const SlotOut *__restrict__ out, int nout, int64_t n_cap,
                               const double *__restrict__ x)
{
    for (int k = blockIdx.x; k < nout; k += gridDim.x) {
        const SlotOut d = out[k];
        for (int64_t e = threadIdx.x; e < 3 * d.n; e += blockDim.x)
            d.lambda[e] = x[3 * d.blob_off + e];
        for (int64_t e = threadIdx.x; e < 6 * d.nb; e += blockDim.x) {
            const int64_t b = e / 6, c = e % 6;
            const double v = x[3 * n_cap + 6 * d.body_off + e];
            if (c < 3) d.U[3 * b + c] = v;
            else d.Omega[3 * b + c - 3] = v;
        }
    }
}

// blob positions of admitted bodies: r_i = q_p + R(theta_p) rho_i
__global__ void eng_blob_kernel(const int64_t *__restrict__ blob_body, int64_t b_lo, int64_t b_hi,
                                const double *__restrict__ q, const double *__restrict__ theta,
                                const double *__restrict__ rho, double *__restrict__ r)
{
    for (int64_t i = b_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b_hi;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = blob_body[i];
        if (p < 0) continue;
        double s = theta[4 * p], x = theta[4 * p + 1], y = theta[4 * p + 2], z = theta[4 * p + 3];
        const double inv = rsqrt(s * s + x * x + y * y + z * z);
        s *= inv; x *= inv; y *= inv; z *= inv;
        const double a = rho[3 * i], b = rho[3 * i + 1], c = rho[3 * i + 2];
        const double d = s * s - (x * x + y * y + z * z);
        const double vr = x * a + y * b + z * c;
        r[3 * i + 0] = q[3 * p + 0] + d * a + 2.0 * x * vr + 2.0 * s * (y * c - z * b);
        r[3 * i + 1] = q[3 * p + 1] + d * b + 2.0 * y * vr + 2.0 * s * (z * a - x * c);
        r[3 * i + 2] = q[3 * p + 2] + d * c + 2.0 * z * vr + 2.0 * s * (x * b - y * a);
    }
}

__global__ void eng_pack_kernel(const double *__restrict__ r, int64_t b_lo, int64_t b_hi,
                                float4 *__restrict__ hi, float4 *__restrict__ lo)
{
    for (int64_t i = b_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b_hi;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = r[3 * i], y = r[3 * i + 1], z = r[3 * i + 2];
        const float xh = (float)x, yh = (float)y, zh = (float)z;
        hi[i] = make_float4(xh, yh, zh, 0.f);
        lo[i] = make_float4((float)(x - (double)xh), (float)(y - (double)yh),
                            (float)(z - (double)zh), 0.f);
    }
}

// b = [slip ; -(F, T)], x = 0 and y_M = 0 on the segments of admitted slots
__global__ void eng_rhs_kernel(const Seg *__restrict__ segs, int nseg, int64_t n_cap,
                               const double *__restrict__ slip, const double *__restrict__ F,
                               const double *__restrict__ T, double *__restrict__ b,
                               double *__restrict__ x, double *__restrict__ ym)
{
    for (int it = blockIdx.x; it < nseg; it += gridDim.x) {
        const Seg sg = segs[it];
        for (int64_t e = sg.start + threadIdx.x; e < sg.end; e += blockDim.x) {
            if (e < 3 * n_cap) {
                b[e] = slip[e];
                ym[e] = 0.0;
            } else {
                const int64_t k = e - 3 * n_cap, p = k / 6, c = k % 6;
                b[e] = c < 3 ? -F[3 * p + c] : -T[3 * p + c - 3];
            }
            x[e] = 0.0;
        }
    }
}

// ------------------------------------------------------------------ pair kernels
template <bool WALL, int NP>
__global__ void __launch_bounds__(kNT, NP == 1 ? 3 : 2) eng_x2_kernel(
    const Work *__restrict__ W, const int64_t *__restrict__ item_off, int nw, int64_t n_items,
    const int *__restrict__ mask, PairConsts2 k, double scale)
{
    __shared__ float4 sP[kX2SmemFloat4PerSource * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const Work P = W[find_owner(item_off, nw, item)];
        if (!mask[P.slot]) continue;  // uniform across the CTA
        const int64_t local = item - P.item_off;
        const int tb = (int)(local % P.n_tblocks);
        const int64_t sc = local / P.n_tblocks;
        const int64_t j0 = sc * P.chunk, j1 = j0 + P.chunk < P.n ? j0 + P.chunk : P.n;
        x2_item<WALL, NP, kNT>(sP, P.hi, P.lo, P.n, P.hi, P.lo, P.f, tb, j0, j1, k,
                               P.S == 1 ? P.y : P.part + 3 * sc * P.n, P.S == 1 ? scale : 1.0);
    }
}

// Symmetric packed pair kernel over every listed request's block-pair
// triangle (blocks of 2*kNT blobs); item -> request -> (I, J); results are
// added to y with FP64 atomics (y zeroed beforehand).  n_tblocks holds the
// request's block count.
template <bool WALL>
__global__ void __launch_bounds__(kNT, 2) eng_sym_kernel(
    const Work *__restrict__ W, const int64_t *__restrict__ item_off, int nw, int64_t n_items,
    const int *__restrict__ mask, PairConsts2 k, double scale)
{
    __shared__ float4 sP[kX2SmemFloat4PerSource * kNT];
    __shared__ float sRev[3 * kNT * (kNT / 32)];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const Work P = W[find_owner(item_off, nw, item)];
        if (!mask[P.slot]) continue;
        const int64_t local = item - P.item_off + P.tri_lo;
        const int64_t nb = P.n_tblocks;
        int64_t lo_r = 0, hi_r = nb;
        while (hi_r - lo_r > 1) {
            const int64_t mid = (lo_r + hi_r) >> 1;
            if (mid * nb - mid * (mid - 1) / 2 <= local) lo_r = mid;
            else hi_r = mid;
        }
        const int64_t I = lo_r, J = I + (local - (I * nb - I * (I - 1) / 2));
        x2sym_item<WALL, kNT>(sP, sRev, P.hi, P.lo, P.f, P.n, I, J, k, P.y, scale);
    }
}

// y = 0 on the listed rows (RSeg work index -> that entry's y)
__global__ void eng_zero_kernel(const Work *__restrict__ W, const RSeg *__restrict__ rs, int nrs,
                                const int *__restrict__ mask)
{
    for (int it = blockIdx.x; it < nrs; it += gridDim.x) {
        const RSeg R = rs[it];
        const Work P = W[R.work];
        if (!mask[P.slot]) continue;
        for (int64_t e = R.start + threadIdx.x; e < R.end; e += blockDim.x) P.y[e] = 0.0;
    }
}

// Symmetric double-float kernel over every listed request's block-pair
// triangle (blocks of kNT blobs); y zeroed beforehand; n_tblocks holds the
// request's block count.
template <bool WALL>
__global__ void __launch_bounds__(kNT) eng_df_kernel(const Work *__restrict__ W,
                                                     const int64_t *__restrict__ item_off, int nw,
                                                     int64_t n_items, const int *__restrict__ mask,
                                                     PairConsts<dfl> k, double scale)
{
    __shared__ float4 sD[3 * kNT];
    __shared__ double sRev[3 * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const Work P = W[find_owner(item_off, nw, item)];
        if (!mask[P.slot]) continue;
        const int64_t local = item - P.item_off;
        const int64_t nb = P.n_tblocks;
        int64_t lo_r = 0, hi_r = nb;
        while (hi_r - lo_r > 1) {
            const int64_t mid = (lo_r + hi_r) >> 1;
            if (mid * nb - mid * (mid - 1) / 2 <= local) lo_r = mid;
            else hi_r = mid;
        }
        const int64_t I = lo_r, J = I + (local - (I * nb - I * (I - 1) / 2));
        dfsym_item<WALL, kNT>(sD, sRev, P.hi, P.lo, P.f, P.n, I, J, k, P.y, scale);
    }
}

template <bool WALL>
__global__ void __launch_bounds__(kNT) eng_f64_kernel(const Work *__restrict__ W,
                                                      const int64_t *__restrict__ item_off, int nw,
                                                      int64_t n_items, const int *__restrict__ mask,
                                                      PairConsts<double> k, double scale)
{
    __shared__ double sm[6 * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const Work P = W[find_owner(item_off, nw, item)];
        if (!mask[P.slot]) continue;
        const int64_t local = item - P.item_off;
        const int tb = (int)(local % P.n_tblocks);
        const int64_t sc = local / P.n_tblocks;
        const int64_t j0 = sc * P.chunk, j1 = j0 + P.chunk < P.n ? j0 + P.chunk : P.n;
        f64_item<WALL, kNT>(sm, P.r, P.n, P.r, P.f, tb, j0, j1, k,
                            P.S == 1 ? P.y : P.part + 3 * sc * P.n, P.S == 1 ? scale : 1.0);
    }
}

// y = scale * sum_s partial[s] for work entries with S > 1
__global__ void eng_reduce_kernel(const Work *__restrict__ W, const RSeg *__restrict__ rs, int nrs,
                                  const int *__restrict__ mask, double scale)
{
    for (int it = blockIdx.x; it < nrs; it += gridDim.x) {
        const RSeg R = rs[it];
        const Work P = W[R.work];
        if (!mask[P.slot] || P.S == 1) continue;
        for (int64_t e = R.start + threadIdx.x; e < R.end; e += blockDim.x) {
            double acc = 0.0;
            for (int s = 0; s < P.S; ++s) acc += P.part[3 * s * P.n + e];
            P.y[e] = scale * acc;
        }
    }
}

// ------------------------------------------------------------------ kinematics
// v_i (+)= alpha * (U_p + Omega_p x (r_i - q_p)) for blobs of masked slots;
// in/out vectors chosen per slot: base + k[slot] * ld
__global__ void eng_K_kernel(const int64_t *__restrict__ blob_body, const int *__restrict__ blob_slot,
                             int64_t b_lo, int64_t b_hi, const double *__restrict__ r,
                             const double *__restrict__ q, const double *in_base,
                             const int *__restrict__ kin, double *out_base,
                             const int *__restrict__ kout, int64_t ld, int64_t n_cap,
                             const int *__restrict__ mask, double alpha, double beta)
{
    for (int64_t i = b_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < b_hi;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int s = blob_slot[i];
        if (s < 0 || !mask[s]) continue;
        const int64_t p = blob_body[i];
        const double *u = in_base + (kin ? kin[s] : 0) * ld + 3 * n_cap + 6 * p;
        double *v = out_base + (kout ? kout[s] : 0) * ld + 3 * i;
        const double dx = r[3 * i] - q[3 * p], dy = r[3 * i + 1] - q[3 * p + 1],
                     dz = r[3 * i + 2] - q[3 * p + 2];
        const double vx = u[0] + (u[4] * dz - u[5] * dy);
        const double vy = u[1] + (u[5] * dx - u[3] * dz);
        const double vz = u[2] + (u[3] * dy - u[4] * dx);
        v[0] = alpha * vx + beta * v[0];
        v[1] = alpha * vy + beta * v[1];
        v[2] = alpha * vz + beta * v[2];
    }
}

// FT_p = alpha * (sum lambda_i, sum (r_i - q_p) x lambda_i) for bodies of masked slots
__global__ void eng_KT_kernel(const int *__restrict__ body_slot, const int64_t *__restrict__ body_b0,
                              const int64_t *__restrict__ body_b1, int64_t p_lo, int64_t p_hi,
                              const double *__restrict__ r, const double *__restrict__ q,
                              const double *in_base, const int *__restrict__ kin, double *out_base,
                              const int *__restrict__ kout, int64_t ld, int64_t n_cap,
                              const int *__restrict__ mask, double alpha)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t p = p_lo + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); p < p_hi;
         p += warps) {
        const int s = body_slot[p];
        if (s < 0 || !mask[s]) continue;
        const double *lam = in_base + (kin ? kin[s] : 0) * ld;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
        for (int64_t i = body_b0[p] + lane; i < body_b1[p]; i += 32) {
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
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o);
        if (lane < 6) {
            double v = acc[0];
#pragma unroll
            for (int c = 1; c < 6; ++c)
                if (lane == c) v = acc[c];
            (out_base + (kout ? kout[s] : 0) * ld)[3 * n_cap + 6 * p + lane] = alpha * v;
        }
    }
}

// Z_{j_s} = P^-1 V_{j_s} body by body for slots doing an Arnoldi step
__global__ void __launch_bounds__(256) eng_precond_apply_kernel(
    const int *__restrict__ body_slot, const int64_t *__restrict__ body_b0,
    const int64_t *__restrict__ body_b1, const int64_t *__restrict__ poff, int64_t p_lo,
    int64_t p_hi, const double *__restrict__ P, const double *__restrict__ V, double *__restrict__ Z,
    const int *__restrict__ jidx, int64_t ld, int64_t n_cap, const int *__restrict__ mask)
{
    extern __shared__ double xs[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t p = p_lo + blockIdx.x; p < p_hi; p += gridDim.x) {
        const int s = body_slot[p];
        if (s < 0 || !mask[s]) continue;  // uniform across the CTA
        const int64_t b0 = body_b0[p];
        const int n = 3 * (int)(body_b1[p] - b0);
        const int m = n + 6;
        const double *v = V + (int64_t)jidx[s] * ld;
        double *z = Z + (int64_t)jidx[s] * ld;
        __syncthreads();
        for (int e = threadIdx.x; e < m; e += blockDim.x)
            xs[e] = e < n ? v[3 * b0 + e] : v[3 * n_cap + 6 * p + (e - n)];
        __syncthreads();
        const double *Pp = P + poff[p];
        for (int row = warp; row < m; row += nw) {
            const double *pr = Pp + (size_t)row * m;
            double acc = 0.0;
            for (int c = lane; c < m; c += 32) acc += pr[c] * xs[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) {
                if (row < n) z[3 * b0 + row] = acc;
                else z[3 * n_cap + 6 * p + (row - n)] = acc;
            }
        }
    }
}

// ------------------------------------------------------------------ Krylov vector kernels
// partial[k * nseg + it] = X_k . w over segment it for k < nk_s = nk_of[s] + nk_add
// (X_k at X + (xk[s] + k)*ld, w at W + wk[s]*ld; null offset arrays mean 0 and
// null nk_of means one vector); masked slots only
__global__ void eng_multidot_kernel(const double *__restrict__ X, const int *__restrict__ xk,
                                    int64_t ld, const int *__restrict__ nk_of, int nk_add,
                                    const double *__restrict__ Wb, const int *__restrict__ wk,
                                    const Seg *__restrict__ segs, int nseg,
                                    const int *__restrict__ mask, double *__restrict__ partial)
{
    __shared__ double red[kRT / 32];
    const int k = blockIdx.y;
    for (int it = blockIdx.x; it < nseg; it += gridDim.x) {
        const Seg sg = segs[it];
        double acc = 0.0;
        const int s = sg.slot;
        const int nk = nk_of ? nk_of[s] + nk_add : 1;
        if (mask[s] && k < nk) {
            const double *x = X + ((xk ? (int64_t)xk[s] : 0) + k) * ld;
            const double *w = Wb + (wk ? (int64_t)wk[s] * ld : 0);
            for (int64_t e = sg.start + threadIdx.x; e < sg.end; e += blockDim.x) acc += x[e] * w[e];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            acc = threadIdx.x < kRT / 32 ? red[threadIdx.x] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (threadIdx.x == 0) partial[(int64_t)k * nseg + it] = acc;
        }
    }
}

// out_s[k] = sum of slot s's segments (fixed order); seg ranges per list entry
__global__ void eng_finish_dots_kernel(const double *__restrict__ partial, int nseg, int nk_max,
                                       const int *__restrict__ list, const int *__restrict__ seg_off,
                                       int nlist, const int *__restrict__ nk_of, int nk_add,
                                       const int *__restrict__ mask, double *__restrict__ sm,
                                       int64_t stride, int64_t off)
{
    const int lane = threadIdx.x & 31;
    const int warps = (blockDim.x >> 5) * gridDim.x;
    for (int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nlist * nk_max;
         w += warps) {
        const int li = w / nk_max, k = w % nk_max;
        const int s = list[li];
        if (!mask[s] || k >= (nk_of ? nk_of[s] + nk_add : 1)) continue;
        double acc = 0.0;
        for (int it = seg_off[li] + lane; it < seg_off[li + 1]; it += 32)
            acc += partial[(int64_t)k * nseg + it];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) sm[(int64_t)s * stride + off + k] = acc;
    }
}

// w_s -= sum_{k < nk_s} V_k h_s[k]   (w at V + (j_s+1)*ld)
__global__ void eng_subtract_kernel(const double *__restrict__ V, int64_t ld,
                                    const int *__restrict__ jidx, const double *__restrict__ sm,
                                    int64_t stride, int64_t h_off, const Seg *__restrict__ segs,
                                    int nseg, const int *__restrict__ mask)
{
    for (int it = blockIdx.x; it < nseg; it += gridDim.x) {
        const Seg sg = segs[it];
        const int s = sg.slot;
        if (!mask[s]) continue;
        const int j = jidx[s];
        const double *h = sm + (int64_t)s * stride + h_off;
        double *w = const_cast<double *>(V) + (int64_t)(j + 1) * ld;
        for (int64_t e = sg.start + threadIdx.x; e < sg.end; e += blockDim.x) {
            double acc = w[e];
            for (int k = 0; k <= j; ++k) acc -= V[(int64_t)k * ld + e] * h[k];
            w[e] = acc;
        }
    }
}

// y = x / sqrt(nrm2_s) on segments; x at X + xk[s]*ld, y at Y + yk[s]*ld
__global__ void eng_normalise_kernel(const double *X, const int *__restrict__ xk, double *Y,
                                     const int *__restrict__ yk, int64_t ld,
                                     const double *__restrict__ sm, int64_t stride, int64_t nrm_off,
                                     const Seg *__restrict__ segs, int nseg,
                                     const int *__restrict__ mask)
{
    for (int it = blockIdx.x; it < nseg; it += gridDim.x) {
        const Seg sg = segs[it];
        const int s = sg.slot;
        if (!mask[s]) continue;
        const double d = sqrt(sm[(int64_t)s * stride + nrm_off]);
        const double inv = d > 0.0 ? 1.0 / d : 0.0;
        const double *x = X + (xk ? (int64_t)xk[s] * ld : 0);
        double *y = Y + (yk ? (int64_t)yk[s] * ld : 0);
        for (int64_t e = sg.start + threadIdx.x; e < sg.end; e += blockDim.x) y[e] = x[e] * inv;
    }
}

// w = b - t on segments of masked slots (or w = b where first[s])
__global__ void eng_residual_kernel(const double *__restrict__ b, const double *__restrict__ t,
                                    double *__restrict__ w, const Seg *__restrict__ segs, int nseg,
                                    const int *__restrict__ resid)
{
    for (int it = blockIdx.x; it < nseg; it += gridDim.x) {
        const Seg sg = segs[it];
        const bool sub = resid[sg.slot] != 0;
        for (int64_t e = sg.start + threadIdx.x; e < sg.end; e += blockDim.x)
            w[e] = sub ? b[e] - t[e] : b[e];
    }
}

// dx = sum_{k < kstep_s} Z_k y_s[k] and x += dx for slots that ended their
// cycle (dx may be null: x only)
__global__ void eng_update_kernel(const double *__restrict__ Z, int64_t ld,
                                  const double *__restrict__ sm, int64_t stride, int64_t y_off,
                                  const int *__restrict__ jidx, const Seg *__restrict__ segs,
                                  int nseg, const int *__restrict__ park, double *__restrict__ x,
                                  double *__restrict__ dx)
{
    for (int it = blockIdx.x; it < nseg; it += gridDim.x) {
        const Seg sg = segs[it];
        const int s = sg.slot;
        if (!park[s]) continue;
        const int nk = jidx[s];
        const double *y = sm + (int64_t)s * stride + y_off;
        for (int64_t e = sg.start + threadIdx.x; e < sg.end; e += blockDim.x) {
            double acc = 0.0;
            for (int k = 0; k < nk; ++k) acc += Z[(int64_t)k * ld + e] * y[k];
            x[e] += acc;
            if (dx) dx[e] = acc;
        }
    }
}

// y_M += t and t = y_M on the blob segments of masked slots
__global__ void eng_accumulate_kernel(double *__restrict__ t, double *__restrict__ ym,
                                      const Seg *__restrict__ segs, int nseg,
                                      const int *__restrict__ mask)
{
    for (int it = blockIdx.x; it < nseg; it += gridDim.x) {
        const Seg sg = segs[it];
        if (!mask[sg.slot]) continue;
        for (int64_t e = sg.start + threadIdx.x; e < sg.end; e += blockDim.x) {
            const double v = ym[e] + t[e];
            ym[e] = v;
            t[e] = v;
        }
    }
}

// out[s] = a[s] && b[s] for every slot
__global__ void eng_and_kernel(const int *__restrict__ a, const int *__restrict__ b,
                               int *__restrict__ out, int n)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        out[s] = a[s] && b[s];
}

// ------------------------------------------------------------------ per-slot scalar kernels
__global__ void eng_init_kernel(const int *__restrict__ list, int nlist, double *sm, SL L,
                                SlotState st)
{
    for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nlist; li += gridDim.x * blockDim.x) {
        const int s = list[li];
        double *q = sm + (int64_t)s * L.total();
        q[L.bnorm()] = sqrt(q[L.nrm2()]);
        const bool zero = !(q[L.bnorm()] > 0.0);
        st.act[s] = 0;
        st.live[s] = zero ? 0 : 1;
        st.conv[s] = zero ? 1 : 0;
        st.j[s] = 0;
        st.iters[s] = 0;
        st.restarts[s] = 0;
        st.park[s] = 0;
        st.fine[s] = 0;
        q[L.rel()] = 0.0;
    }
}

// After the true residual norms: finish, or start a cycle (act = 1, j = 0).
__global__ void eng_cycle_start_kernel(const int *__restrict__ list, int nlist, double *sm, SL L,
                                       SlotState st, double tol, int maxit, int mixed)
{
    for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nlist; li += gridDim.x * blockDim.x) {
        const int s = list[li];
        st.park[s] = 0;
        st.act[s] = 0;
        st.j[s] = 0;
        if (!st.live[s]) continue;
        double *q = sm + (int64_t)s * L.total();
        const double beta = sqrt(q[L.nrm2()]);
        const double rel = beta / q[L.bnorm()];
        q[L.rel()] = rel;
        st.fine[s] = mixed && rel <= kFineRel * tol;
        if (rel <= tol) {
            st.conv[s] = 1;
            st.live[s] = 0;
            continue;
        }
        if (rel != rel || st.iters[s] >= maxit) {
            st.live[s] = 0;
            continue;
        }
        for (int i = 0; i <= L.m; ++i) q[L.g() + i] = 0.0;
        q[L.g()] = beta;
        q[L.est()] = beta;
        double inner = 0.5 * tol * q[L.bnorm()];
        if (mixed) inner = fmax(inner, 1e-5 * beta);
        q[L.inner()] = inner;
        st.act[s] = 1;
    }
}

// Column j_s: merge the CGS passes, rotate, update g; end the cycle when the
// estimate meets the target, the iteration budget is spent or the basis is full.
__global__ void eng_givens_kernel(const int *__restrict__ list, int nlist, double *sm, SL L,
                                  SlotState st, int maxit)
{
    for (int li = blockIdx.x * blockDim.x + threadIdx.x; li < nlist; li += gridDim.x * blockDim.x) {
        const int s = list[li];
        if (!st.act[s]) continue;
        const int j = st.j[s];
        double *q = sm + (int64_t)s * L.total();
        for (int i = 0; i <= j; ++i) q[L.H(i, j)] = q[L.h() + i] + q[L.y() + i];
        q[L.H(j + 1, j)] = sqrt(q[L.nrm2()]);
        for (int i = 0; i < j; ++i) {
            const double c = q[L.cs() + i], sn = q[L.sn() + i];
            const double a = q[L.H(i, j)], b = q[L.H(i + 1, j)];
            q[L.H(i, j)] = c * a + sn * b;
            q[L.H(i + 1, j)] = -sn * a + c * b;
        }
        const double a = q[L.H(j, j)], b = q[L.H(j + 1, j)];
        const double rr = hypot(a, b);
        const double c = rr > 0.0 ? a / rr : 1.0;
        const double sn = rr > 0.0 ? b / rr : 0.0;
        q[L.cs() + j] = c;
        q[L.sn() + j] = sn;
        q[L.H(j, j)] = rr;
        q[L.H(j + 1, j)] = 0.0;
        const double gj = q[L.g() + j];
        q[L.g() + j] = c * gj;
        q[L.g() + j + 1] = -sn * gj;
        q[L.est()] = fabs(sn * gj);
        st.iters[s] += 1;
        st.j[s] = j + 1;
        if (!(q[L.est()] > q[L.inner()]) || st.iters[s] >= maxit || j + 1 >= L.m) {
            st.act[s] = 0;
            st.park[s] = 1;
            // back substitution R y = g (j + 1 columns)
            const int k = j + 1;
            for (int i = k - 1; i >= 0; --i) {
                double acc = q[L.g() + i];
                for (int jj = i + 1; jj < k; ++jj) acc -= q[L.H(i, jj)] * q[L.y() + jj];
                const double d = q[L.H(i, i)];
                q[L.y() + i] = d != 0.0 ? acc / d : 0.0;
            }
            st.restarts[s] += 1;
        }
    }
}

int grid_for(int64_t work, int per) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, per), 8192)); }

// ------------------------------------------------------------------ host-side range allocator
struct RangeAlloc {
    std::map<int64_t, int64_t> free_;  // start -> length
    int64_t cap = 0;
    void init(int64_t c)
    {
        cap = c;
        free_.clear();
        if (c > 0) free_[0] = c;
    }
    int64_t alloc(int64_t len)
    {
        if (len <= 0) return 0;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                const int64_t s = it->first, rest = it->second - len;
                free_.erase(it);
                if (rest > 0) free_[s + len] = rest;
                return s;
            }
        }
        return -1;
    }
    // longest free range (0 if none)
    int64_t largest() const
    {
        int64_t m = 0;
        for (const auto &kv : free_) m = std::max(m, kv.second);
        return m;
    }
    void release(int64_t s, int64_t len)
    {
        if (len <= 0) return;
        auto it = free_.emplace(s, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace

// ------------------------------------------------------------------ engine
struct Engine {
    mb_context *ctx = nullptr;
    mb_params prm{};
    int m = 1;
    SL L{1};
    int64_t n_cap = 0, b_cap = 0, pc_cap = 0, start_cap = 0;
    int s_cap = 0;
    int64_t ld = 0;  // vector length 3 n_cap + 6 b_cap
    mb::DevBuf arena, partial, scratch, tick, work_buf;
    // device arrays carved from the arena
    double *rho, *r, *slip, *q, *theta, *F, *T, *P;
    float4 *hi, *lo;
    int64_t *bstart, *body_b0, *body_b1, *blob_body, *poff;
    int *blob_slot, *body_slot;
    double *V, *Z, *b, *x, *w, *t, *sm, *dpart;
    double *dx = nullptr, *ym = nullptr;  // mixed: cycle correction, running M lambda
    SlotState st{};
    int *flag = nullptr;
    int *hstate = nullptr;  // pinned mirror of per-slot ints (kSlotInts arrays)
    RangeAlloc blobs, bodies, pcs, starts;
    std::vector<int> free_slots;
    bool mixed = false;
    double tick_pairs = -1;  // per-request pair budget of one tick's Arnoldi matvec (< 0: none)
    int max_bypass = 64;     // admissions that may overtake a queued request (< 0: none)
    int np_variant = 1;     // FP32 tile shape: 1, 2 = packed with 2 or 4 targets per
                            // thread, 3 = symmetric (autotuned)
    std::map<int, int> tuned_by_class;  // autotuned tile shape per size class of a tick's pairs

    struct Req {
        int64_t ticket = 0;
        mb_problem prob{};
        std::vector<int64_t> hstart;
        int slot = -1;
        int64_t blob_off = -1, body_off = -1, pc_off = -1, start_off = -1, pc_len = 0;
        int max_np = 1;  // most blobs on one body
        int phase = 0;  // 0 queued, 1 first cycle, 2 residual, 3 arnoldi, 4 done
        int j = 0;
        int mv_chunks = 1, mv_next = 0;  // split of the current Arnoldi matvec
        clk::time_point t_submit, t_admit, t_done;
        mb_info info{};
        int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
        mb_status err = MB_OK;
        int bypassed = 0;  // later requests admitted while this one waited
    };
    std::deque<Req *> queue;
    std::deque<int64_t> finished;            // tickets retired since the last mb_server_finished
    std::vector<Req *> running;              // by slot
    std::map<int64_t, Req *> all;            // ticket -> request
    int64_t next_ticket = 1;

    ~Engine()
    {
        for (auto &kv : all) delete kv.second;
        release(ctx, arena);
        release(ctx, partial);
        release(ctx, scratch);
        release(ctx, tick);
        release(ctx, work_buf);
        if (hstate) cudaFreeHost(hstate);
    }

    mb_status create(mb_context *c, const mb_params *p, int64_t max_blobs, int64_t max_bodies,
                     int64_t max_pc_doubles, int max_requests, double tick_pair_budget = -1,
                     int bypass_limit = 64)
    {
        ctx = c;
        prm = *p;
        tick_pairs = tick_pair_budget;
        max_bypass = bypass_limit;
        m = std::max(1, std::min(p->restart, 500));
        L = SL{m};
        n_cap = max_blobs;
        b_cap = max_bodies;
        pc_cap = max_pc_doubles;
        s_cap = max_requests;
        start_cap = max_bodies + max_requests;
        ld = 3 * n_cap + 6 * b_cap;
        mixed = p->prec == MB_MIXED_REFINE;
        size_t need = 0;
        auto add = [&](size_t bytes) { need += ((bytes + 255) & ~(size_t)255); };
        add(sizeof(double) * 3 * n_cap * 3);                       // rho, r, slip
        add(sizeof(double) * b_cap * 13);                          // q, theta, F, T
        add(sizeof(double) * pc_cap);                              // preconditioner blocks
        add(sizeof(float4) * n_cap * 2);                           // hi, lo
        add(sizeof(int64_t) * (start_cap + 3 * b_cap + n_cap));    // bstart, b0, b1, poff, blob_body
        add(sizeof(int) * (n_cap + b_cap));                        // slots of blobs/bodies
        add(sizeof(double) * ld * (2 * m + 1 + 4));                // V, Z, b, x, w, t
        if (mixed) add(sizeof(double) * (ld + 3 * n_cap));         // dx, y_M
        add(sizeof(double) * L.total() * s_cap);                   // per-slot scalars
        add(sizeof(int) * kSlotInts * s_cap + 64);                 // slot state, flag
        MB_TRY(ensure(ctx, arena, need + 4096, "server arena"));
        char *base = (char *)arena.ptr;
        size_t off = 0;
        auto take = [&](size_t bytes) {
            off = (off + 255) & ~(size_t)255;
            void *p = base + off;
            off += bytes;
            return p;
        };
        rho = (double *)take(sizeof(double) * 3 * n_cap);
        r = (double *)take(sizeof(double) * 3 * n_cap);
        slip = (double *)take(sizeof(double) * 3 * n_cap);
        q = (double *)take(sizeof(double) * 3 * b_cap);
        theta = (double *)take(sizeof(double) * 4 * b_cap);
        F = (double *)take(sizeof(double) * 3 * b_cap);
        T = (double *)take(sizeof(double) * 3 * b_cap);
        P = (double *)take(sizeof(double) * pc_cap);
        hi = (float4 *)take(sizeof(float4) * n_cap);
        lo = (float4 *)take(sizeof(float4) * n_cap);
        bstart = (int64_t *)take(sizeof(int64_t) * start_cap);
        body_b0 = (int64_t *)take(sizeof(int64_t) * b_cap);
        body_b1 = (int64_t *)take(sizeof(int64_t) * b_cap);
        poff = (int64_t *)take(sizeof(int64_t) * b_cap);
        blob_body = (int64_t *)take(sizeof(int64_t) * n_cap);
        blob_slot = (int *)take(sizeof(int) * n_cap);
        body_slot = (int *)take(sizeof(int) * b_cap);
        V = (double *)take(sizeof(double) * ld * (m + 1));
        Z = (double *)take(sizeof(double) * ld * m);
        b = (double *)take(sizeof(double) * ld);
        x = (double *)take(sizeof(double) * ld);
        w = (double *)take(sizeof(double) * ld);
        t = (double *)take(sizeof(double) * ld);
        if (mixed) {
            dx = (double *)take(sizeof(double) * ld);
            ym = (double *)take(sizeof(double) * 3 * n_cap);
        }
        sm = (double *)take(sizeof(double) * L.total() * s_cap);
        int *ints = (int *)take(sizeof(int) * kSlotInts * s_cap);
        flag = (int *)take(sizeof(int) * 16);
        st = SlotState{ints, ints + s_cap, ints + 2 * s_cap, ints + 3 * s_cap, ints + 4 * s_cap,
                       ints + 5 * s_cap, ints + 6 * s_cap, ints + 7 * s_cap, ints + 8 * s_cap};
        MB_CUDA_TRY(ctx, cudaMemset(blob_slot, 0xff, sizeof(int) * n_cap));
        MB_CUDA_TRY(ctx, cudaMemset(body_slot, 0xff, sizeof(int) * b_cap));
        MB_CUDA_TRY(ctx, cudaMemset(blob_body, 0xff, sizeof(int64_t) * n_cap));
        MB_CUDA_TRY(ctx, cudaMemset(ints, 0, sizeof(int) * kSlotInts * s_cap));
        MB_CUDA_TRY(ctx, cudaMallocHost(&hstate, sizeof(int) * kSlotInts * s_cap + 64));
        blobs.init(n_cap);
        bodies.init(b_cap);
        pcs.init(pc_cap);
        starts.init(start_cap);
        running.assign(s_cap, nullptr);
        free_slots.clear();
        for (int s = s_cap - 1; s >= 0; --s) free_slots.push_back(s);
        return MB_OK;
    }

    mb_status submit(const mb_problem &pr, int64_t *ticket)
    {
        if (pr.n_bodies <= 0 || pr.n_blobs <= 0 || !pr.q || !pr.theta || !pr.blob_start || !pr.rho ||
            !pr.F || !pr.T || !pr.U || !pr.Omega || !pr.lambda)
            return set_err(ctx, MB_EINVAL, "malformed request");
        Req *rq = new (std::nothrow) Req();
        if (!rq) return MB_ENOMEM;
        rq->prob = pr;
        rq->hstart.resize(pr.n_bodies + 1);
        cudaError_t e = cudaMemcpy(rq->hstart.data(), pr.blob_start,
                                   sizeof(int64_t) * (pr.n_bodies + 1), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            delete rq;
            return cuda_err(ctx, e, "reading blob_start");
        }
        int64_t pc = 0;
        for (int64_t p = 0; p < pr.n_bodies; ++p) {
            const int64_t np = rq->hstart[p + 1] - rq->hstart[p];
            if (np < 1 || rq->hstart[0] != 0 || rq->hstart[pr.n_bodies] != pr.n_blobs) {
                delete rq;
                return set_err(ctx, MB_EINVAL,
                               "blob_start must start at 0, end at N and give every body a blob");
            }
            pc += (3 * np + 6) * (3 * np + 6);
            rq->max_np = std::max<int>(rq->max_np, (int)np);
        }
        rq->pc_len = pc;
        if (pr.n_blobs > n_cap || pr.n_bodies > b_cap || pc > pc_cap) {
            delete rq;
            return set_err(ctx, MB_ENOMEM, "request larger than the server's arena");
        }
        rq->ticket = next_ticket++;
        rq->t_submit = clk::now();
        queue.push_back(rq);
        all[rq->ticket] = rq;
        *ticket = rq->ticket;
        return MB_OK;
    }

    // ------------------------------------------------------------ tick helpers
    void segs_of(const Req *rq, std::vector<Seg> &out, bool blobs_part = true, bool bodies_part = true)
    {
        const int64_t ranges[2][2] = {{3 * rq->blob_off, 3 * (rq->blob_off + rq->prob.n_blobs)},
                                      {3 * n_cap + 6 * rq->body_off,
                                       3 * n_cap + 6 * (rq->body_off + rq->prob.n_bodies)}};
        for (int k = 0; k < 2; ++k) {
            if ((k == 0 && !blobs_part) || (k == 1 && !bodies_part)) continue;
            for (int64_t a = ranges[k][0]; a < ranges[k][1]; a += kSeg)
                out.push_back(Seg{a, std::min(ranges[k][1], a + kSeg), rq->slot, 0});
        }
    }

    // Upload a small host array into the per-tick buffer; returns device pointer.
    template <typename Tt>
    Tt *upload(const std::vector<Tt> &v, size_t &off, cudaStream_t s, mb_status *st_out)
    {
        off = (off + 255) & ~(size_t)255;
        Tt *d = (Tt *)((char *)tick.ptr + off);
        off += sizeof(Tt) * std::max<size_t>(1, v.size());
        if (!v.empty()) {
            cudaError_t e = cudaMemcpyAsync(d, v.data(), sizeof(Tt) * v.size(),
                                            cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) *st_out = cuda_err(ctx, e, "tick upload");
        }
        return d;
    }

    // Batched pair matvec over `list` slots: y_s = M f_s, f and y at vector
    // slots (fk, yk) of the arena's vector arrays.
    // tri (symmetric FP32 only): per list entry, the range [lo, hi) of the
    // request's block-pair items to evaluate (a part of a split matvec);
    // zero_mask: requests whose output is zeroed first (default: mask).
    mb_status matvec(const std::vector<int> &list, const double *f_base, const std::vector<int64_t> &fk,
                     double *y_base, const std::vector<int64_t> &yk, mb_precision prec,
                     const int *mask, cudaStream_t s, size_t &toff,
                     const std::vector<std::pair<int64_t, int64_t>> *tri = nullptr,
                     const int *zero_mask = nullptr)
    {
        if (list.empty()) return MB_OK;
        const double scale = 1.0 / (6.0 * kPi * prm.eta * prm.a);
        const bool x2 = prec == MB_FP32_KAHAN;
        const bool dfs = prec == MB_DF64;          // symmetric double-float
        const bool sym = (x2 && np_variant == 3) || dfs;
        const int tpc = x2 ? 2 * (np_variant == 3 ? 1 : np_variant) * kNT : kNT;
        int occ = 1;
        if (dfs)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_df_kernel<true>, kNT, 0);
        else if (sym)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_sym_kernel<true>, kNT, 0);
        else if (prec == MB_FP32_KAHAN)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_x2_kernel<true, 1>, kNT, 0);
        else if (prec == MB_DF64)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_df_kernel<true>, kNT, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, eng_f64_kernel<true>, kNT, 0);
        const int res = std::max(1, occ) * ctx->sm_count;
        double pairs = 0;
        for (int sl : list) pairs += (double)running[sl]->prob.n_blobs * running[sl]->prob.n_blobs;
        int64_t chunk = (int64_t)std::ceil(pairs / (8.0 * res) / tpc / kNT) * kNT;
        chunk = std::max<int64_t>(chunk, 2 * kNT);
        std::vector<Work> W;
        std::vector<int64_t> ioff;
        std::vector<RSeg> rs;
        int64_t items = 0, part = 0;
        for (size_t li = 0; li < list.size(); ++li) {
            const Req *rq = running[list[li]];
            Work wk{};
            wk.n = rq->prob.n_blobs;
            wk.hi = hi + rq->blob_off;
            wk.lo = lo + rq->blob_off;
            wk.r = r + 3 * rq->blob_off;
            wk.f = f_base + fk[li] * ld + 3 * rq->blob_off;
            wk.y = y_base + yk[li] * ld + 3 * rq->blob_off;
            wk.slot = rq->slot;
            wk.item_off = items;
            ioff.push_back(items);
            if (sym) {
                const int64_t nb = ceil_div(wk.n, tpc);
                wk.n_tblocks = (int)nb;
                wk.S = 1;
                wk.chunk = wk.n;
                wk.tri_lo = 0;
                int64_t cnt = nb * (nb + 1) / 2;
                if (tri && x2) {
                    wk.tri_lo = (int)(*tri)[li].first;
                    cnt = (*tri)[li].second - (*tri)[li].first;
                }
                items += cnt;
                for (int64_t a = 0; a < 3 * wk.n; a += kSeg)
                    rs.push_back(RSeg{a, std::min<int64_t>(3 * wk.n, a + kSeg), (int)li, 0});
                W.push_back(wk);
                continue;
            }
            wk.n_tblocks = (int)ceil_div(wk.n, tpc);
            int S = (int)std::max<int64_t>(1, ceil_div(wk.n, chunk));
            wk.chunk = ceil_div(ceil_div(wk.n, S), kNT) * kNT;
            wk.S = (int)ceil_div(wk.n, wk.chunk);
            items += (int64_t)wk.n_tblocks * wk.S;
            if (wk.S > 1) {
                wk.part = (double *)0 + part;  // offset, fixed up below
                for (int64_t a = 0; a < 3 * wk.n; a += kSeg)
                    rs.push_back(RSeg{a, std::min<int64_t>(3 * wk.n, a + kSeg), (int)li, 0});
                part += 3 * wk.n * wk.S;
            }
            W.push_back(wk);
        }
        ioff.push_back(items);
        MB_TRY(ensure(ctx, partial, sizeof(double) * std::max<int64_t>(1, part), "server partials"));
        for (auto &wk : W)
            if (wk.S > 1) wk.part = (double *)partial.ptr + (wk.part - (double *)0);
        mb_status stt = MB_OK;
        Work *dW = upload(W, toff, s, &stt);
        int64_t *dI = upload(ioff, toff, s, &stt);
        RSeg *dR = upload(rs, toff, s, &stt);
        MB_TRY(stt);
        const int nw = (int)W.size();
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, res));
        const bool wall = prm.wall != 0;
        auto *ev = profile_begin(ctx, s);
        if (sym) {
            eng_zero_kernel<<<grid_for((int64_t)rs.size(), 1), 256, 0, s>>>(
                dW, dR, (int)rs.size(), zero_mask ? zero_mask : mask);
            count_launch();
        }
        if (dfs) {
            const PairConsts<dfl> k = PairConsts<dfl>::make(prm.a);
            if (wall) eng_df_kernel<true><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
            else eng_df_kernel<false><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
        } else if (sym) {
            const PairConsts2 k = PairConsts2::make(prm.a);
            if (wall) eng_sym_kernel<true><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
            else eng_sym_kernel<false><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
        } else if (prec == MB_FP32_KAHAN) {
            const PairConsts2 k = PairConsts2::make(prm.a);
            if (np_variant == 1) {
                if (wall) eng_x2_kernel<true, 1><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
                else eng_x2_kernel<false, 1><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
            } else {
                if (wall) eng_x2_kernel<true, 2><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
                else eng_x2_kernel<false, 2><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
            }
        } else {
            const PairConsts<double> k = PairConsts<double>::make(prm.a);
            if (wall) eng_f64_kernel<true><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
            else eng_f64_kernel<false><<<grid, kNT, 0, s>>>(dW, dI, nw, items, mask, k, scale);
        }
        profile_end(ev, s);
        count_launch();
        if (!rs.empty() && !sym) {
            eng_reduce_kernel<<<grid_for((int64_t)rs.size(), 1), 256, 0, s>>>(dW, dR, (int)rs.size(),
                                                                           mask, scale);
            count_launch();
        }
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }

    // dots over the segments of `list` slots; results to sm[s*stride + off + k]
    mb_status dots(const std::vector<int> &list, const std::vector<Seg> &segs,
                   const std::vector<int> &seg_off, const double *X, const int *xk,
                   const int *nk_of, int nk_add, int nk_max, const double *Wb, const int *wk,
                   const int *mask, int64_t off, cudaStream_t s, size_t &toff)
    {
        if (segs.empty()) return MB_OK;
        mb_status stt = MB_OK;
        const Seg *dS = upload(segs, toff, s, &stt);
        const int *dL = upload(list, toff, s, &stt);
        const int *dO = upload(seg_off, toff, s, &stt);
        MB_TRY(stt);
        MB_TRY(ensure_dpart((int64_t)segs.size() * nk_max));
        const int nseg = (int)segs.size();
        eng_multidot_kernel<<<dim3(std::min(nseg, 8192), nk_max), kRT, 0, s>>>(
            X, xk, ld, nk_of, nk_add, Wb, wk, dS, nseg, mask, dpart);
        count_launch();
        const int warps = (int)list.size() * nk_max;
        eng_finish_dots_kernel<<<(int)ceil_div(warps, 8), 256, 0, s>>>(
            dpart, nseg, nk_max, dL, dO, (int)list.size(), nk_of, nk_add, mask, sm, L.total(), off);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }
    mb::DevBuf dpart_buf;
    mb_status ensure_dpart(int64_t n)
    {
        MB_TRY(ensure(ctx, dpart_buf, sizeof(double) * std::max<int64_t>(1, n), "server dot partials"));
        dpart = (double *)dpart_buf.ptr;
        return MB_OK;
    }

    mb_status step(cudaStream_t s, int *n_running, int *n_queued);
    mb_status retire(Req *rq, int conv, int iters, int restarts, cudaStream_t s);
};

mb_status Engine::step(cudaStream_t s, int *n_running, int *n_queued)
{
    MB_TRY(ensure(ctx, tick, (size_t)16 << 20, "server tick buffer"));
    size_t toff = 0;
    mb_status stt = MB_OK;
    const mb_precision inner = inner_precision(prm.prec);
    const mb_precision outer = outer_precision(prm.prec);

    // ---- 1. admission: scan the queue in arrival order and admit every
    // request whose ranges fit.  Requests that do not fit stay queued in
    // order; each admission behind one counts as a bypass, and a request
    // bypassed max_bypass times ends the scan (nothing behind it is admitted
    // until it is), so its wait is bounded by the requests ahead of it
    // finishing.  max_bypass < 0 gives strict first-come first-served.
    std::vector<Req *> admitted;
    int64_t big_b = blobs.largest(), big_p = bodies.largest(), big_c = pcs.largest(),
            big_s = starts.largest();
    std::vector<Req *> waiting;  // queued requests passed over in this scan
    for (auto it = queue.begin(); it != queue.end() && !free_slots.empty();) {
        Req *rq = *it;
        int64_t bo = -1, po = -1, co = -1, so = -1;
        const bool may_fit = rq->prob.n_blobs <= big_b && rq->prob.n_bodies <= big_p &&
                             rq->pc_len <= big_c && rq->prob.n_bodies + 1 <= big_s;
        if (may_fit && (bo = blobs.alloc(rq->prob.n_blobs)) >= 0) {
            if ((po = bodies.alloc(rq->prob.n_bodies)) < 0) {
                blobs.release(bo, rq->prob.n_blobs);
            } else if ((co = pcs.alloc(rq->pc_len)) < 0) {
                blobs.release(bo, rq->prob.n_blobs);
                bodies.release(po, rq->prob.n_bodies);
            } else if ((so = starts.alloc(rq->prob.n_bodies + 1)) < 0) {
                blobs.release(bo, rq->prob.n_blobs);
                bodies.release(po, rq->prob.n_bodies);
                pcs.release(co, rq->pc_len);
            }
        }
        if (so < 0) {  // does not fit now
            if (max_bypass < 0 || rq->bypassed >= max_bypass) break;
            waiting.push_back(rq);
            ++it;
            continue;
        }
        it = queue.erase(it);
        for (Req *w : waiting) ++w->bypassed;
        big_b = blobs.largest();
        big_p = bodies.largest();
        big_c = pcs.largest();
        big_s = starts.largest();
        rq->blob_off = bo; rq->body_off = po; rq->pc_off = co; rq->start_off = so;
        rq->slot = free_slots.back();
        free_slots.pop_back();
        rq->phase = 1;
        rq->j = 0;
        rq->state = 1;
        rq->t_admit = clk::now();
        running[rq->slot] = rq;
        admitted.push_back(rq);
    }
    if (!admitted.empty()) {
        std::vector<SlotIn> in;
        std::vector<int> slots;
        std::vector<int64_t> hpoff;
        for (Req *rq : admitted) {
            const mb_problem &p = rq->prob;
            in.push_back(SlotIn{p.q, p.theta, p.rho, p.F, p.T, p.slip, p.blob_start, p.n_blobs,
                                p.n_bodies, rq->blob_off, rq->body_off, rq->start_off});
            slots.push_back(rq->slot);
        }
        SlotIn *dIn = upload(in, toff, s, &stt);
        int *dSl = upload(slots, toff, s, &stt);
        MB_TRY(stt);
        admit_kernel<<<(int)admitted.size(), 256, 0, s>>>(dIn, (int)admitted.size(), dSl, rho, slip,
                                                          q, theta, F, T, bstart, body_b0, body_b1,
                                                          blob_slot, body_slot, blob_body, st.bad);
        count_launch();
        for (Req *rq : admitted) {
            const int64_t b0 = rq->blob_off, b1 = rq->blob_off + rq->prob.n_blobs;
            eng_blob_kernel<<<grid_for(b1 - b0, 256), 256, 0, s>>>(blob_body, b0, b1, q, theta, rho, r);
            eng_pack_kernel<<<grid_for(b1 - b0, 256), 256, 0, s>>>(r, b0, b1, hi, lo);
            count_launch(2);
            // preconditioner offsets of this request's bodies in the P range
            std::vector<int64_t> po(rq->prob.n_bodies);
            int64_t acc = rq->pc_off;
            for (int64_t p = 0; p < rq->prob.n_bodies; ++p) {
                po[p] = acc;
                const int64_t np = rq->hstart[p + 1] - rq->hstart[p];
                acc += (3 * np + 6) * (3 * np + 6);
            }
            MB_CUDA_TRY(ctx, cudaMemcpyAsync(poff + rq->body_off, po.data(),
                                             sizeof(int64_t) * po.size(), cudaMemcpyHostToDevice, s));
            // the copy reads a host vector: make it complete before it goes out of scope
            MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            int max_np = 0;
            for (int64_t p = 0; p < rq->prob.n_bodies; ++p)
                max_np = std::max<int>(max_np, (int)(rq->hstart[p + 1] - rq->hstart[p]));
            MB_TRY(precond_setup_range(ctx, rq->prob.n_bodies, r, q + 3 * rq->body_off,
                                       bstart + rq->start_off, poff + rq->body_off, P, max_np,
                                       prm.a, prm.eta, prm.wall, st.bad, rq->slot, s));
        }
        std::vector<Seg> segs;
        std::vector<int> seg_off, list;
        for (Req *rq : admitted) {
            seg_off.push_back((int)segs.size());
            segs_of(rq, segs);
            list.push_back(rq->slot);
        }
        seg_off.push_back((int)segs.size());
        Seg *dS = upload(segs, toff, s, &stt);
        MB_TRY(stt);
        eng_rhs_kernel<<<grid_for((int64_t)segs.size(), 1), 256, 0, s>>>(dS, (int)segs.size(), n_cap,
                                                                         slip, F, T, b, x, ym ? ym : t);
        count_launch();
        // b.b per admitted slot, then initial state; the admitted slots act
        // as the mask (live is not set yet): use a temporary all-ones mask
        std::vector<int> ones(s_cap, 0);
        for (int sl : list) ones[sl] = 1;
        int *dOnes = upload(ones, toff, s, &stt);
        int *dList = upload(list, toff, s, &stt);
        MB_TRY(stt);
        MB_TRY(dots(list, segs, seg_off, b, nullptr, nullptr, 0, 1, b, nullptr, dOnes, L.nrm2(), s,
                    toff));
        eng_init_kernel<<<1, 128, 0, s>>>(dList, (int)list.size(), sm, L, st);
        count_launch();
        std::vector<int> hbad(s_cap, 0);
        MB_CUDA_TRY(ctx, cudaMemcpyAsync(hbad.data(), st.bad, sizeof(int) * s_cap,
                                         cudaMemcpyDeviceToHost, s));
        MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        toff = 0;  // uploads above have completed
        for (Req *rq : admitted) {
            const int bd = hbad[rq->slot];
            if (!bd) continue;
            // malformed descriptor or non-positive-definite block: fail the request now
            rq->state = 3;
            rq->err = bd == 1 ? MB_EINVAL : MB_ESINGULAR;
            rq->phase = 4;
            const int zero = 0;
            MB_CUDA_TRY(ctx, cudaMemcpy(st.live + rq->slot, &zero, sizeof(int), cudaMemcpyHostToDevice));
            MB_TRY(retire(rq, 0, 0, 0, s));
        }
    }

    // ---- which slots do what this tick
    std::vector<int> cyc, resid_list;     // starting a cycle; of those, needing b - A x
    std::vector<int> arn;                 // doing an Arnoldi step (may include cyc)
    for (int sl = 0; sl < s_cap; ++sl) {
        Req *rq = running[sl];
        if (!rq || rq->phase == 4) continue;
        if (rq->phase == 1 || rq->phase == 2) cyc.push_back(sl);
        if (rq->phase == 2) resid_list.push_back(sl);
        arn.push_back(sl);
    }
    if (arn.empty()) {
        *n_running = 0;
        *n_queued = (int)queue.size();
        return MB_OK;
    }
    // tile shape: the context's pinned pair variant if any (the scalar
    // variant maps to packed x2), else autotuned once per size class of the
    // tick's pair work (powers of 4): small ticks favour the packed shapes,
    // large ones the symmetric shape.  It stays fixed while a split matvec is
    // in progress, since only the symmetric shape splits.
    bool mid_split = false, tune = false;
    double tick_pair_sum = 0;
    for (int sl : arn) {
        const Req *rq = running[sl];
        tick_pair_sum += (double)rq->prob.n_blobs * rq->prob.n_blobs;
        mid_split = mid_split || (rq->phase == 3 && rq->mv_next > 0);
    }
    const int size_class = (int)(std::log2(std::max(1.0, tick_pair_sum)) / 2);
    if (inner == MB_FP32_KAHAN && ctx->pair_variant >= 0) {
        np_variant = std::min(3, std::max(1, ctx->pair_variant));
    } else if (inner == MB_FP32_KAHAN && !mid_split) {
        auto it = tuned_by_class.find(size_class);
        if (it != tuned_by_class.end()) np_variant = it->second;
        else tune = true;
    }
    if (tune) {
        float best = 1e30f;
        int best_v = 1;
        cudaEvent_t e0, e1;
        MB_CUDA_TRY(ctx, cudaEventCreate(&e0));
        MB_CUDA_TRY(ctx, cudaEventCreate(&e1));
        // time the candidates on every 8th active request (the size mix of
        // the whole list at an eighth of its pair work), all of them when few
        std::vector<int> sample;
        for (size_t i = 0; i < arn.size(); i += (arn.size() >= 16 ? 8 : 1)) sample.push_back(arn[i]);
        std::vector<int64_t> zk(sample.size(), 0);
        std::vector<int> ones(s_cap, 0);
        for (int sl : sample) ones[sl] = 1;
        for (int cand = 1; cand <= 3; ++cand) {
            np_variant = cand;
            size_t off2 = 0;
            int *dm = upload(ones, off2, s, &stt);
            MB_TRY(stt);
            MB_CUDA_TRY(ctx, cudaEventRecord(e0, s));
            MB_TRY(matvec(sample, b, zk, t, zk, MB_FP32_KAHAN, dm, s, off2));
            MB_CUDA_TRY(ctx, cudaEventRecord(e1, s));
            MB_CUDA_TRY(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            MB_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_v = cand; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        np_variant = best_v;
        tuned_by_class[size_class] = best_v;
        toff = 0;
    }

    // ---- 2. true residuals and cycle starts
    if (!cyc.empty()) {
        std::vector<int> rmask(s_cap, 0);
        for (int sl : resid_list) rmask[sl] = 1;
        int *dR = upload(rmask, toff, s, &stt);
        MB_TRY(stt);
        if (!resid_list.empty() && mixed) {
            // t = y_M += M dx, the product in FP32 for slots whose cycle
            // started small enough (fine), else in the outer precision
            std::vector<int> lf, lc, mf(s_cap, 0), mc(s_cap, 0);
            for (int sl : resid_list) {
                if (hstate[8 * s_cap + sl]) { lf.push_back(sl); mf[sl] = 1; }
                else { lc.push_back(sl); mc[sl] = 1; }
            }
            int *dMf = upload(mf, toff, s, &stt);
            int *dMc = upload(mc, toff, s, &stt);
            MB_TRY(stt);
            std::vector<int64_t> zf(lf.size(), 0), zc(lc.size(), 0);
            MB_TRY(matvec(lf, dx, zf, t, zf, inner, dMf, s, toff));
            MB_TRY(matvec(lc, dx, zc, t, zc, outer, dMc, s, toff));
            std::vector<Seg> bsegs;
            for (int sl : resid_list) segs_of(running[sl], bsegs, true, false);
            Seg *dB = upload(bsegs, toff, s, &stt);
            MB_TRY(stt);
            eng_accumulate_kernel<<<grid_for((int64_t)bsegs.size(), 1), 256, 0, s>>>(
                t, ym, dB, (int)bsegs.size(), dR);
            count_launch();
        } else if (!resid_list.empty()) {
            std::vector<int64_t> zero(resid_list.size(), 0);
            MB_TRY(matvec(resid_list, x, zero, t, zero, outer, dR, s, toff));
        }
        if (!resid_list.empty()) {
            eng_K_kernel<<<grid_for(n_cap, 256), 256, 0, s>>>(blob_body, blob_slot, 0, n_cap, r, q, x,
                                                              nullptr, t, nullptr, ld, n_cap, dR,
                                                              -1.0, 1.0);
            eng_KT_kernel<<<grid_for(b_cap * 32, 256), 256, 0, s>>>(body_slot, body_b0, body_b1, 0,
                                                                    b_cap, r, q, x, nullptr, t,
                                                                    nullptr, ld, n_cap, dR, -1.0);
            count_launch(2);
        }
        std::vector<Seg> segs;
        std::vector<int> seg_off;
        for (int sl : cyc) {
            seg_off.push_back((int)segs.size());
            segs_of(running[sl], segs);
        }
        seg_off.push_back((int)segs.size());
        Seg *dS = upload(segs, toff, s, &stt);
        int *dC = upload(cyc, toff, s, &stt);
        MB_TRY(stt);
        eng_residual_kernel<<<grid_for((int64_t)segs.size(), 1), 256, 0, s>>>(b, t, w, dS,
                                                                             (int)segs.size(), dR);
        count_launch();
        MB_TRY(dots(cyc, segs, seg_off, w, nullptr, nullptr, 0, 1, w, nullptr, st.live, L.nrm2(), s,
                    toff));
        eng_cycle_start_kernel<<<1, 128, 0, s>>>(dC, (int)cyc.size(), sm, L, st, prm.tol,
                                                 prm.maxit, mixed);
        count_launch();
        eng_normalise_kernel<<<grid_for((int64_t)segs.size(), 1), 256, 0, s>>>(
            w, nullptr, V, nullptr, ld, sm, L.total(), L.nrm2(), dS, (int)segs.size(), st.act);
        count_launch();
    }

    // ---- 3. one Arnoldi step for every active slot
    {
        std::vector<int64_t> zk, vk;
        int jmax = 0;
        for (int sl : arn) {
            const int j = (running[sl]->phase == 3) ? running[sl]->j : 0;
            zk.push_back(j);
            vk.push_back(j + 1);
            jmax = std::max(jmax, j);
        }
        std::vector<Seg> segs;
        std::vector<int> seg_off;
        for (int sl : arn) {
            seg_off.push_back((int)segs.size());
            segs_of(running[sl], segs);
        }
        seg_off.push_back((int)segs.size());
        // Split matvecs: with the symmetric FP32 tile shape, a request whose
        // matvec exceeds tick_pairs evaluations does it in parts over
        // consecutive ticks (the kernel accumulates into its zeroed output).
        // The preconditioner apply, the zeroing and K / K^T run on the first
        // part's tick, the orthogonalisation and Givens update on the last's.
        const bool can_split = tick_pairs > 0 && inner == MB_FP32_KAHAN && np_variant == 3;
        std::vector<int> first(s_cap, 0), last(s_cap, 0), arn_last;
        std::vector<std::pair<int64_t, int64_t>> tri;
        for (int sl : arn) {
            Req *rq = running[sl];
            const int64_t nblk = ceil_div(rq->prob.n_blobs, 2 * (int64_t)kNT);
            const int64_t items = nblk * (nblk + 1) / 2;
            if (rq->phase != 3 || rq->mv_next == 0) {
                const double pairs = 0.5 * (double)rq->prob.n_blobs * rq->prob.n_blobs;
                rq->mv_chunks = can_split
                                    ? (int)std::min<double>((double)items,
                                                            std::max(1.0, std::ceil(pairs / tick_pairs)))
                                    : 1;
                rq->mv_next = 0;
            }
            const int c = rq->mv_next, C = rq->mv_chunks;
            first[sl] = c == 0;
            last[sl] = c == C - 1;
            tri.emplace_back(items * c / C, items * (c + 1) / C);
            if (last[sl]) arn_last.push_back(sl);
        }
        Seg *dS = upload(segs, toff, s, &stt);
        int *dA = upload(arn_last, toff, s, &stt);
        int *dFirst = upload(first, toff, s, &stt);
        int *dLast = upload(last, toff, s, &stt);
        MB_TRY(stt);
        // device masks: active and on the first / last part of its matvec
        int *act_first = (int *)((char *)tick.ptr + ((toff + 255) & ~(size_t)255));
        toff = ((toff + 255) & ~(size_t)255) + sizeof(int) * s_cap;
        int *act_last = (int *)((char *)tick.ptr + ((toff + 255) & ~(size_t)255));
        toff = ((toff + 255) & ~(size_t)255) + sizeof(int) * s_cap;
        eng_and_kernel<<<grid_for(s_cap, 256), 256, 0, s>>>(st.act, dFirst, act_first, s_cap);
        eng_and_kernel<<<grid_for(s_cap, 256), 256, 0, s>>>(st.act, dLast, act_last, s_cap);
        count_launch(2);
        // precond apply for bodies of active slots: Z_j = P^-1 V_j
        int max_np = 1;
        for (int sl : arn) max_np = std::max(max_np, running[sl]->max_np);
        const int pc_smem = (int)sizeof(double) * (3 * max_np + 6);
        const int pc_grid = (int)std::min<int64_t>(b_cap, 8 * (int64_t)ctx->sm_count);
        eng_precond_apply_kernel<<<pc_grid, 256, pc_smem, s>>>(body_slot, body_b0, body_b1, poff, 0,
                                                               b_cap, P, V, Z, st.j, ld, n_cap,
                                                               act_first);
        count_launch();
        MB_TRY(matvec(arn, Z, zk, V, vk, inner, st.act, s, toff, &tri, act_first));
        eng_K_kernel<<<grid_for(n_cap, 256), 256, 0, s>>>(blob_body, blob_slot, 0, n_cap, r, q, Z,
                                                          st.j, V + ld, st.j, ld, n_cap, act_first,
                                                          -1.0, 1.0);
        count_launch();
        // K^T writes -K^T z into V_{j+1}: output slot index j+1 via a shifted view
        eng_KT_kernel<<<grid_for(b_cap * 32, 256), 256, 0, s>>>(body_slot, body_b0, body_b1, 0, b_cap,
                                                                r, q, Z, st.j, V + ld, st.j, ld,
                                                                n_cap, act_first, -1.0);
        count_launch();
        // CGS2: h = V^T w, w -= V h, twice; |w|; normalise (w = V_{j+1})
        const int nk = jmax + 1;
        MB_TRY(dots(arn, segs, seg_off, V, nullptr, st.j, 1, nk, V + ld, st.j, act_last, L.h(), s,
                    toff));
        eng_subtract_kernel<<<grid_for((int64_t)segs.size(), 1), 256, 0, s>>>(
            V, ld, st.j, sm, L.total(), L.h(), dS, (int)segs.size(), act_last);
        count_launch();
        MB_TRY(dots(arn, segs, seg_off, V, nullptr, st.j, 1, nk, V + ld, st.j, act_last, L.y(), s,
                    toff));
        eng_subtract_kernel<<<grid_for((int64_t)segs.size(), 1), 256, 0, s>>>(
            V, ld, st.j, sm, L.total(), L.y(), dS, (int)segs.size(), act_last);
        count_launch();
        MB_TRY(dots(arn, segs, seg_off, V + ld, st.j, nullptr, 0, 1, V + ld, st.j, act_last,
                    L.nrm2(), s, toff));
        eng_normalise_kernel<<<grid_for((int64_t)segs.size(), 1), 256, 0, s>>>(
            V + ld, st.j, V + ld, st.j, ld, sm, L.total(), L.nrm2(), dS, (int)segs.size(), act_last);
        count_launch();
        eng_givens_kernel<<<1, 128, 0, s>>>(dA, (int)arn_last.size(), sm, L, st, prm.maxit);
        count_launch();
        eng_update_kernel<<<grid_for((int64_t)segs.size(), 1), 256, 0, s>>>(
            Z, ld, sm, L.total(), L.y(), st.j, dS, (int)segs.size(), st.park, x, dx);
        count_launch();
        (void)dA;
    }
    MB_CUDA_TRY(ctx, cudaGetLastError());

    // ---- 4. read the slot state back; retire finished requests
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(hstate, st.act, sizeof(int) * kSlotInts * s_cap,
                                     cudaMemcpyDeviceToHost, s));
    MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const int *h_act = hstate, *h_live = hstate + s_cap, *h_park = hstate + 6 * s_cap,
              *h_j = hstate + 3 * s_cap;
    std::vector<Req *> finished;
    for (int sl : arn) {
        Req *rq = running[sl];
        if (!h_live[sl]) {
            rq->phase = 4;
            finished.push_back(rq);
        } else if (h_park[sl]) {
            rq->phase = 2;
            rq->j = 0;
            rq->mv_next = 0;
        } else if (h_act[sl]) {
            rq->phase = 3;
            rq->j = h_j[sl];
            // a split matvec continues on the next tick; a finished step starts anew
            rq->mv_next = rq->mv_next + 1 < rq->mv_chunks ? rq->mv_next + 1 : 0;
        } else {
            rq->phase = 2;  // defensive: restart from the true residual
        }
    }
    for (Req *rq : finished) {
        const int sl = rq->slot;
        MB_TRY(retire(rq, hstate[2 * s_cap + sl], hstate[4 * s_cap + sl], hstate[5 * s_cap + sl], s));
    }
    int nr = 0;
    for (Req *rq : running)
        if (rq) ++nr;
    *n_running = nr;
    *n_queued = (int)queue.size();
    return MB_OK;
}

// Write a finished request's results to its arrays (unless it failed),
// return its ranges and slot to the free lists, and record its info.
mb_status Engine::retire(Req *rq, int conv, int iters, int restarts, cudaStream_t s)
{
    const int sl = rq->slot;
    double rel = 0.0;
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(&rel, sm + (int64_t)sl * L.total() + L.rel(), sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
    SlotOut o{rq->prob.U, rq->prob.Omega, rq->prob.lambda, rq->prob.n_blobs, rq->prob.n_bodies,
              rq->blob_off, rq->body_off};
    SlotOut *dO = (SlotOut *)tick.ptr;  // retire runs after the tick's uploads completed
    MB_CUDA_TRY(ctx, cudaMemcpyAsync(dO, &o, sizeof(SlotOut), cudaMemcpyHostToDevice, s));
    if (rq->state != 3) {
        scatter_kernel<<<1, 256, 0, s>>>(dO, 1, n_cap, x);
        count_launch();
    }
    release_kernel<<<1, 256, 0, s>>>(dO, 1, blob_slot, body_slot, blob_body);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    MB_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    rq->t_done = clk::now();
    if (rq->state == 3) {
        rq->info = mb_info{};
    } else {
        rq->state = 2;
        rq->info.iters = iters;
        rq->info.restarts = restarts;
        rq->info.converged = conv;
        rq->info.rel_residual = rel;
        if (!conv) rq->err = MB_ENOTCONVERGED;
    }
    rq->info.setup_ms = std::chrono::duration<double, std::milli>(rq->t_admit - rq->t_submit).count();
    rq->info.solve_ms = std::chrono::duration<double, std::milli>(rq->t_done - rq->t_admit).count();
    blobs.release(rq->blob_off, rq->prob.n_blobs);
    bodies.release(rq->body_off, rq->prob.n_bodies);
    pcs.release(rq->pc_off, rq->pc_len);
    starts.release(rq->start_off, rq->prob.n_bodies + 1);
    running[sl] = nullptr;
    free_slots.push_back(sl);
    rq->slot = -1;
    finished.push_back(rq->ticket);
    return MB_OK;
}

mb_status solve_batch(mb_context *ctx, int np, const mb_problem *probs, const mb_params *prm,
                      mb_info *infos, cudaStream_t s)
{
    int64_t nt = 0, bt = 0, pct = 0;
    std::vector<std::vector<int64_t>> hs(np);
    for (int p = 0; p < np; ++p) {
        nt += probs[p].n_blobs;
        bt += probs[p].n_bodies;
        hs[p].resize(probs[p].n_bodies + 1);
        MB_CUDA_TRY(ctx, cudaMemcpy(hs[p].data(), probs[p].blob_start,
                                    sizeof(int64_t) * (probs[p].n_bodies + 1), cudaMemcpyDeviceToHost));
        for (int64_t b = 0; b < probs[p].n_bodies; ++b) {
            const int64_t k = hs[p][b + 1] - hs[p][b];
            if (k > 0) pct += (3 * k + 6) * (3 * k + 6);
        }
    }
    Engine *E = new (std::nothrow) Engine();
    if (!E) return MB_ENOMEM;
    mb_status st = E->create(ctx, prm, nt, bt, std::max<int64_t>(1, pct), np);
    std::vector<int64_t> tickets(np, 0);
    for (int p = 0; p < np && st == MB_OK; ++p) {
        st = E->submit(probs[p], &tickets[p]);
        if (st != MB_OK) {
            const std::string m = ctx->err;
            st = set_err(ctx, st, "problem %d: %s", p, m.c_str());
        }
    }
    int nr = 1, nq = 1;
    while (st == MB_OK && (nr > 0 || nq > 0)) st = E->step(s, &nr, &nq);
    mb_status result = st;
    int n_bad = 0;
    if (st == MB_OK) {
        for (int p = 0; p < np; ++p) {
            Engine::Req *rq = E->all[tickets[p]];
            if (infos) infos[p] = rq->info;
            if (rq->err == MB_EINVAL || rq->err == MB_ESINGULAR) {
                if (result == MB_OK)
                    result = set_err(ctx, rq->err,
                                     rq->err == MB_EINVAL
                                         ? "problem %d: blob_start[0] must be 0 and blob_start[n_b] = N"
                                         : "problem %d: a body's mobility block is not positive definite",
                                     p);
            } else if (rq->err == MB_ENOTCONVERGED) {
                ++n_bad;
            }
        }
        if (result == MB_OK && n_bad)
            result = set_err(ctx, MB_ENOTCONVERGED, "%d of %d problems did not converge within maxit",
                             n_bad, np);
    }
    delete E;
    return result;
}

}  // namespace mb

struct mb_server {
    mb::Engine eng;
};

using namespace mb;

extern "C" {

mb_status mb_server_create(mb_context *ctx, const mb_params *params,
                           const mb_server_limits *limits, mb_server **server)
{
    if (!ctx || !params || !limits || !server) return MB_EINVAL;
    *server = nullptr;
    ctx->err.clear();
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_err(ctx, MB_ECUDA, "cudaSetDevice");
    if (!(params->a > 0.0) || !(params->eta > 0.0) || !(params->tol > 0.0) || params->maxit < 1 ||
        params->restart < 1 || params->prec < MB_FP64 || params->prec > MB_DF64)
        return set_err(ctx, MB_EINVAL, "bad solver parameters");
    if (params->precond != MB_PRECOND_WALL)
        return set_err(ctx, MB_EINVAL, "the serving engine uses MB_PRECOND_WALL only");
    if (limits->max_blobs < 1 || limits->max_bodies < 1 || limits->max_precond_bytes < 8 ||
        limits->max_requests < 1 || limits->max_requests > (1 << 20))
        return set_err(ctx, MB_EINVAL, "bad server limits");
    mb_server *sv = new (std::nothrow) mb_server();
    if (!sv) return MB_ENOMEM;
    const double budget = limits->tick_pairs == 0.0 ? 1e9 : limits->tick_pairs;
    const int bypass = limits->max_bypass == 0 ? 64 : limits->max_bypass;
    mb_status st = sv->eng.create(ctx, params, limits->max_blobs, limits->max_bodies,
                                  limits->max_precond_bytes / 8, limits->max_requests, budget,
                                  bypass);
    if (st != MB_OK) {
        delete sv;
        return st;
    }
    *server = sv;
    return MB_OK;
}

mb_status mb_server_destroy(mb_server *server)
{
    if (!server) return MB_EINVAL;
    cudaSetDevice(server->eng.ctx->device);
    cudaDeviceSynchronize();
    delete server;
    return MB_OK;
}

mb_status mb_server_submit(mb_server *server, const mb_problem *problem, int64_t *ticket)
{
    if (!server || !problem || !ticket) return MB_EINVAL;
    server->eng.ctx->err.clear();
    return server->eng.submit(*problem, ticket);
}

mb_status mb_server_step(mb_server *server, void *stream, int *n_running, int *n_queued)
{
    if (!server) return MB_EINVAL;
    int nr = 0, nq = 0;
    server->eng.ctx->err.clear();
    if (cudaSetDevice(server->eng.ctx->device) != cudaSuccess) return MB_ECUDA;
    mb_status st = server->eng.step((cudaStream_t)stream, &nr, &nq);
    if (n_running) *n_running = nr;
    if (n_queued) *n_queued = nq;
    return st;
}

mb_status mb_server_finished(mb_server *server, int64_t *tickets, int max_tickets, int *count)
{
    if (!server || !count || max_tickets < 0 || (max_tickets > 0 && !tickets)) return MB_EINVAL;
    auto &fin = server->eng.finished;
    int k = 0;
    while (k < max_tickets && !fin.empty()) {
        tickets[k++] = fin.front();
        fin.pop_front();
    }
    *count = k;
    return MB_OK;
}

mb_status mb_server_poll(mb_server *server, int64_t ticket, int *state, mb_info *info,
                         mb_status *result)
{
    if (!server) return MB_EINVAL;
    auto it = server->eng.all.find(ticket);
    if (it == server->eng.all.end()) return set_err(server->eng.ctx, MB_EINVAL, "unknown ticket");
    const Engine::Req *rq = it->second;
    if (state) *state = rq->state;
    if (info) *info = rq->info;
    if (result) *result = rq->err;
    return MB_OK;
}

}  // extern "C"
