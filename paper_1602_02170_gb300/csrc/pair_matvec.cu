// O(N^2) direct-summation product u = M f of the wall-corrected RPY blob
// mobility (Section 2.1.1; Section 5 evaluates it by direct summation on a
// GPU).
//
// Work decomposition: targets are cut into blocks of NT * TPT blobs (one CTA,
// TPT targets per thread) and sources into S chunks; a persistent grid of one
// wave of CTAs walks the (target block, source chunk) items.  Each CTA stages
// NT sources at a time in shared memory (coalesced float4 loads; every thread
// then reads the same source, a shared-memory broadcast) and accumulates the
// tile in FP32 registers, folding each tile sum into a Kahan-compensated
// accumulator.  Chunk partials go to an FP64 buffer that a second kernel sums
// in a fixed order, so results are deterministic.
//
// FP32 positions carry a hi/lo split: d = (hi_i - hi_j) + (lo_i - lo_j); the
// hi difference is exact for nearby blobs (Sterbenz), so near pairs keep full
// FP32 accuracy even at |x| of several hundred.
#include <algorithm>
#include <mutex>

#include "mb_internal.cuh"
#include "pair_tiles.cuh"
#include "rpy_wall.cuh"

namespace mb {
namespace {

#ifndef MB_PAIR_NT
#define MB_PAIR_NT 256
#endif
#ifndef MB_PAIR_TPT
#define MB_PAIR_TPT 1
#endif
constexpr int kNT = MB_PAIR_NT;   // threads per CTA = sources per shared tile
constexpr double kPi = 3.14159265358979323846;

// Coordinates as unsigned integers in the order of the floats (for min/max).
__device__ __forceinline__ unsigned float_order(float x)
{
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float order_float(unsigned u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Block-wide min of v[0..2] and max of v[3..5] (up to 32 warps; red holds
// 6 x 32) into out[0..5]; every thread of the block must call it.
__device__ __forceinline__ void minmax_block(unsigned (&v)[6], unsigned *red, unsigned *out)
{
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned t = __shfl_xor_sync(0xffffffffu, v[c], o);
            v[c] = c < 3 ? min(v[c], t) : max(v[c], t);
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) red[6 * (threadIdx.x >> 5) + c] = v[c];
    __syncthreads();
    if (threadIdx.x < 6) {
        const int c = threadIdx.x;
        unsigned r = red[c];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            r = c < 3 ? min(r, red[6 * w + c]) : max(r, red[6 * w + c]);
        out[c] = r;
    }
    __syncthreads();
}

// Positions split into FP32 hi and lo parts.  BOX: also the CTA's bounding
// box of the hi parts (ordered integers: min x, y, z, max x, y, z) into
// part[6 blockIdx.x ..], for the spatial order.
template <bool BOX>
__global__ void __launch_bounds__(256) pack_hilo_kernel(const double *__restrict__ r, int64_t n,
                                                        float4 *__restrict__ hi,
                                                        float4 *__restrict__ lo,
                                                        unsigned *__restrict__ part)
{
    unsigned v[6] = {~0u, ~0u, ~0u, 0u, 0u, 0u};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double x = r[3 * i], y = r[3 * i + 1], z = r[3 * i + 2];
        const float xh = (float)x, yh = (float)y, zh = (float)z;
        hi[i] = make_float4(xh, yh, zh, 0.f);
        lo[i] = make_float4((float)(x - (double)xh), (float)(y - (double)yh),
                            (float)(z - (double)zh), 0.f);
        if (BOX) {
            const unsigned o[3] = {float_order(xh), float_order(yh), float_order(zh)};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c] = min(v[c], o[c]);
                v[3 + c] = max(v[3 + c], o[c]);
            }
        }
    }
    if (BOX) {
        __shared__ unsigned red[6 * 32], box[6];
        minmax_block(v, red, box);
        if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = box[threadIdx.x];
    }
}

template <bool WALL, int TPT>
__global__ void __launch_bounds__(kNT) pair_f32_kernel(
    const float4 *__restrict__ hi, const float4 *__restrict__ lo, const double *__restrict__ f,
    int64_t n, int64_t chunk, int n_tblocks, int64_t n_items, PairConsts<float> k,
    double *__restrict__ out, double scale, int direct)
{
    __shared__ float4 sA[kNT];  // (x_hi, y_hi, z_hi, f_x)
    __shared__ float4 sB[kNT];  // (x_lo, y_lo, z_lo, f_y)
    __shared__ float sC[kNT];   // f_z

    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tb = (int)(item % n_tblocks);
        const int64_t sc = item / n_tblocks;
        float xh[TPT], yh[TPT], zh[TPT], xl[TPT], yl[TPT], zl[TPT];
        float sx[TPT], sy[TPT], sz[TPT], cx[TPT], cy[TPT], cz[TPT];
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            int64_t i = (int64_t)tb * kNT * TPT + t * kNT + threadIdx.x;
            i = i < n ? i : n - 1;
            const float4 h = hi[i], l = lo[i];
            xh[t] = h.x; yh[t] = h.y; zh[t] = h.z;
            xl[t] = l.x; yl[t] = l.y; zl[t] = l.z;
            sx[t] = sy[t] = sz[t] = cx[t] = cy[t] = cz[t] = 0.f;
        }
        const int64_t j_begin = sc * chunk;
        const int64_t j_end = j_begin + chunk < n ? j_begin + chunk : n;
        for (int64_t jt = j_begin; jt < j_end; jt += kNT) {
            __syncthreads();
            {
                const int64_t j = jt + threadIdx.x;
                const bool valid = j < j_end;
                const int64_t jc = valid ? j : j_begin;
                const float4 h = hi[jc], l = lo[jc];
                const float fx = valid ? (float)f[3 * jc] : 0.f;
                const float fy = valid ? (float)f[3 * jc + 1] : 0.f;
                const float fz = valid ? (float)f[3 * jc + 2] : 0.f;
                sA[threadIdx.x] = make_float4(h.x, h.y, h.z, fx);
                sB[threadIdx.x] = make_float4(l.x, l.y, l.z, fy);
                sC[threadIdx.x] = fz;
            }
            __syncthreads();
            float ax[TPT], ay[TPT], az[TPT];
#pragma unroll
            for (int t = 0; t < TPT; ++t) ax[t] = ay[t] = az[t] = 0.f;
#pragma unroll 4
            for (int s = 0; s < kNT; ++s) {
                const float4 A = sA[s];
                const float4 B = sB[s];
                const float fz = sC[s];
#pragma unroll
                for (int t = 0; t < TPT; ++t) {
                    const float dx = (xh[t] - A.x) + (xl[t] - B.x);
                    const float dy = (yh[t] - A.y) + (yl[t] - B.y);
                    const float dz = (zh[t] - A.z) + (zl[t] - B.z);
                    pair_accumulate<WALL, float>(dx, dy, dz, zh[t], A.z, A.w, B.w, fz, k, ax[t],
                                                 ay[t], az[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < TPT; ++t) {
                kahan_add(sx[t], cx[t], ax[t]);
                kahan_add(sy[t], cy[t], ay[t]);
                kahan_add(sz[t], cz[t], az[t]);
            }
        }
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            const int64_t i = (int64_t)tb * kNT * TPT + t * kNT + threadIdx.x;
            if (i < n) {
                const double vx = (double)sx[t] - (double)cx[t];
                const double vy = (double)sy[t] - (double)cy[t];
                const double vz = (double)sz[t] - (double)cz[t];
                double *o = direct ? out + 3 * i : out + 3 * (sc * n + i);
                const double m = direct ? scale : 1.0;
                o[0] = m * vx;
                o[1] = m * vy;
                o[2] = m * vz;
            }
        }
    }
}

// Packed FP32 kernel (paired f32x2 arithmetic, 2*NP targets per thread): a
// persistent loop over (target block, source chunk) items; see x2_item.
template <bool WALL, int NP, int NT = kNT>
__global__ void __launch_bounds__(NT, NT == kNT ? (NP == 1 ? 3 : 2) : 16) pair_f32x2_kernel(
    const float4 *__restrict__ hi, const float4 *__restrict__ lo, const double *__restrict__ f,
    int64_t n, int64_t chunk, int n_tblocks, int64_t n_items, PairConsts2 k,
    double *__restrict__ out, double scale, int direct)
{
    __shared__ float4 sP[kX2SmemFloat4PerSource * NT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tb = (int)(item % n_tblocks);
        const int64_t sc = item / n_tblocks;
        const int64_t j_begin = sc * chunk;
        const int64_t j_end = j_begin + chunk < n ? j_begin + chunk : n;
        x2_item<WALL, NP, NT>(sP, hi, lo, n, hi, lo, f, tb, j_begin, j_end, k,
                              direct ? out : out + 3 * sc * n, direct ? scale : 1.0);
    }
}

// Symmetric packed kernel: persistent loop over the upper-triangular block
// pairs (I <= J) of blocks of 2*kNT blobs, row by row; see x2sym_item.
//
// box (optional): the bounding box of every block, (min x, y, z, max x, y, z),
// and grid->far2, the squared distance beyond which a block pair is far (see
// x2sym_item); such pairs take the FAR instance.
struct SortGrid {
    float lo[3], inv_h[3];  // cell of x: (x - lo) * inv_h per axis
    int bits[3];            // bits of the cell index per axis (nbits in all)
    float far2;             // squared box distance of a far block pair
};

template <bool WALL>
__global__ void __launch_bounds__(kNT, 2) pair_sym_kernel(
    const float4 *__restrict__ hi, const float4 *__restrict__ lo, const double *__restrict__ f,
    int64_t n, int64_t nb, int64_t n_items, PairConsts2 k, double *__restrict__ u, double scale,
    const float *__restrict__ box, const SortGrid *__restrict__ grid)
{
    __shared__ float4 sP[kX2SmemFloat4PerSource * kNT];
    __shared__ float sRev[3 * kNT * (kNT / 32)];
    const float far2 = box ? fmaxf(grid->far2, 1.5625f * k.four_a2) : 0.f;
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        // row I holds nb - I items; rowoff(I) = I*nb - I*(I-1)/2
        int64_t lo_r = 0, hi_r = nb;
        while (hi_r - lo_r > 1) {
            const int64_t mid = (lo_r + hi_r) >> 1;
            if (mid * nb - mid * (mid - 1) / 2 <= item) lo_r = mid;
            else hi_r = mid;
        }
        const int64_t I = lo_r;
        const int64_t J = I + (item - (I * nb - I * (I - 1) / 2));
        bool far = false;
        if (box && I != J) {
            const float *bi = box + 6 * I, *bj = box + 6 * J;
            float d2 = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float g = fmaxf(fmaxf(bj[c] - bi[3 + c], bi[c] - bj[3 + c]), 0.f);
                d2 = fmaf(g, g, d2);
            }
            far = d2 > far2;  // the same in every thread
        }
        if (far) x2sym_item<WALL, kNT, true>(sP, sRev, hi, lo, f, n, I, J, k, u, scale);
        else x2sym_item<WALL, kNT, false>(sP, sRev, hi, lo, f, n, I, J, k, u, scale);
    }
}

template <bool WALL, int NT = kNT>
__global__ void __launch_bounds__(NT) pair_f64_kernel(
    const double *__restrict__ r, const double *__restrict__ f, int64_t n, int64_t chunk,
    int n_tblocks, int64_t n_items, PairConsts<double> k, double *__restrict__ out, double scale,
    int direct)
{
    __shared__ double sm[6 * NT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tb = (int)(item % n_tblocks);
        const int64_t sc = item / n_tblocks;
        const int64_t j_begin = sc * chunk;
        const int64_t j_end = j_begin + chunk < n ? j_begin + chunk : n;
        f64_item<WALL, NT>(sm, r, n, r, f, tb, j_begin, j_end, k, direct ? out : out + 3 * sc * n,
                           direct ? scale : 1.0);
    }
}

// FP64 kernel for larger problems: symmetric over the upper-triangular
// pairs of blocks of kNT blobs (one target per thread); see f64sym_item.
template <bool WALL>
__global__ void __launch_bounds__(kNT) pair_f64sym_kernel(
    const double *__restrict__ r, const double *__restrict__ f, int64_t n, int64_t nb,
    int64_t n_items, PairConsts<double> k, double *__restrict__ u, double scale)
{
    __shared__ double sm[9 * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        int64_t lo_r = 0, hi_r = nb;
        while (hi_r - lo_r > 1) {
            const int64_t mid = (lo_r + hi_r) >> 1;
            if (mid * nb - mid * (mid - 1) / 2 <= item) lo_r = mid;
            else hi_r = mid;
        }
        const int64_t I = lo_r, J = I + (item - (I * nb - I * (I - 1) / 2));
        f64sym_item<WALL, kNT>(sm, r, f, n, I, J, k, u, scale);
    }
}

// Double-float kernel: symmetric over the upper-triangular pairs of blocks
// of kNT blobs (one target per thread); see dfsym_item.
// Flow evaluation at points other than the blobs (targets != sources):
// packed FP32 and FP64 items over (target block, source chunk), partials
// reduced like the matvec's.  The targets are tracers of the blob radius a
// (Appendix B renders flows with small blobs of radius a').
template <bool WALL>
__global__ void __launch_bounds__(kNT, 3) eval_f32x2_kernel(
    const float4 *__restrict__ thi, const float4 *__restrict__ tlo, int64_t nt,
    const float4 *__restrict__ hi, const float4 *__restrict__ lo, const double *__restrict__ f,
    int64_t ns, int64_t chunk, int n_tblocks, int64_t n_items, PairConsts2 k,
    double *__restrict__ out, double scale, int direct)
{
    __shared__ float4 sP[kX2SmemFloat4PerSource * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tb = (int)(item % n_tblocks);
        const int64_t sc = item / n_tblocks;
        const int64_t j_begin = sc * chunk;
        const int64_t j_end = j_begin + chunk < ns ? j_begin + chunk : ns;
        x2_item<WALL, 1, kNT>(sP, thi, tlo, nt, hi, lo, f, tb, j_begin, j_end, k,
                              direct ? out : out + 3 * sc * nt, direct ? scale : 1.0);
    }
}

template <bool WALL>
__global__ void __launch_bounds__(kNT) eval_f64_kernel(
    const double *__restrict__ x, int64_t nt, const double *__restrict__ r,
    const double *__restrict__ f, int64_t ns, int64_t chunk, int n_tblocks, int64_t n_items,
    PairConsts<double> k, double *__restrict__ out, double scale, int direct)
{
    __shared__ double sm[6 * kNT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tb = (int)(item % n_tblocks);
        const int64_t sc = item / n_tblocks;
        const int64_t j_begin = sc * chunk;
        const int64_t j_end = j_begin + chunk < ns ? j_begin + chunk : ns;
        f64_item<WALL, kNT>(sm, x, nt, r, f, tb, j_begin, j_end, k,
                            direct ? out : out + 3 * sc * nt, direct ? scale : 1.0);
    }
}

// Appendix B: each blob i becomes n_sub blobs at r_i + off_k carrying
// lambda_i / n_sub each (k fastest).
__global__ void refine_blobs_kernel(const double *__restrict__ r, const double *__restrict__ lam,
                                    int64_t n, const double *__restrict__ off, int n_sub,
                                    double *__restrict__ rs, double *__restrict__ ls)
{
    const double w = 1.0 / n_sub;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n_sub;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / n_sub;
        const int k = (int)(e % n_sub);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            rs[3 * e + c] = r[3 * i + c] + off[3 * k + c];
            ls[3 * e + c] = lam[3 * i + c] * w;
        }
    }
}

// Double-float, forward only, for the smallest problems: blocks of kSmallNT
// targets (one per thread) against source chunks of kSmallNT / 2, every
// ordered pair evaluated (the forward half of pair_sym_rg; the reverse half
// is dead code for the compiler), the block's sums added to u (zeroed) with
// FP64 atomics.  Twice the pair evaluations of the symmetric kernel, in
// several times as many one-warp CTAs: a few hundred blobs fill the GPU.
template <bool WALL, int NT>
__global__ void __launch_bounds__(NT) pair_dfx_kernel(
    const float4 *__restrict__ hi, const float4 *__restrict__ lo, const double *__restrict__ f,
    int64_t n, int64_t chunk, int n_tblocks, int64_t n_items, PairConsts<dfl> k,
    double *__restrict__ u, double scale)
{
    __shared__ float4 sD[3 * NT];
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int tb = (int)(item % n_tblocks);
        const int64_t j0 = (item / n_tblocks) * chunk;
        const int64_t j1 = j0 + chunk < n ? j0 + chunk : n;
        const int64_t i = (int64_t)tb * NT + threadIdx.x;
        const int64_t ic = i < n ? i : n - 1;
        const float4 th = hi[ic], tl = lo[ic];
        const dfl xi(th.x, tl.x), yi(th.y, tl.y), zi(th.z, tl.z);
        __syncthreads();  // the previous item is done with sD
        if (j0 + threadIdx.x < j1) {
            const int64_t j = j0 + threadIdx.x;
            const float4 h = hi[j], l = lo[j];
            const dfl fx(f[3 * j]), fy(f[3 * j + 1]), fz(f[3 * j + 2]);
            float4 *d = sD + 3 * threadIdx.x;
            d[0] = make_float4(h.x, l.x, h.y, l.y);
            d[1] = make_float4(h.z, l.z, fx.hi, fx.lo);
            d[2] = make_float4(fy.hi, fy.lo, fz.hi, fz.lo);
        }
        __syncthreads();
        dfl ux, uy, uz, vx, vy, vz;
        const int cnt = (int)(j1 - j0);
        for (int s = 0; s < cnt; ++s) {
            const float4 A = sD[3 * s], B = sD[3 * s + 1], C = sD[3 * s + 2];
            const dfl zj(B.x, B.y);
            pair_sym_rg<WALL, dfl>(xi - dfl(A.x, A.y), yi - dfl(A.z, A.w), zi - zj, zi, zj,
                                   dfl(B.z, B.w), dfl(C.x, C.y), dfl(C.z, C.w), dfl(), dfl(), dfl(),
                                   k, ux, uy, uz, vx, vy, vz);
        }
        if (i < n) {
            atomicAdd(u + 3 * i, scale * to_double(ux));
            atomicAdd(u + 3 * i + 1, scale * to_double(uy));
            atomicAdd(u + 3 * i + 2, scale * to_double(uz));
        }
    }
}

// box (optional, spatial order): the bounding boxes of the sort's blocks of
// 2 kNT blobs (two blocks of this kernel each); block pairs whose boxes are
// 64 a or more apart take the FAR instance of the item.
template <bool WALL, int NT = kNT>
__global__ void __launch_bounds__(NT) pair_df_kernel(
    const float4 *__restrict__ hi, const float4 *__restrict__ lo, const double *__restrict__ f,
    int64_t n, int64_t nb, int64_t n_items, PairConsts<dfl> k, double *__restrict__ u,
    double scale, const float *__restrict__ box, float far2)
{
    __shared__ float4 sD[3 * NT];
    __shared__ double sRev[3 * NT];
    constexpr int kPer = 2 * kNT / NT;  // this kernel's blocks per box
    for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
        int64_t lo_r = 0, hi_r = nb;
        while (hi_r - lo_r > 1) {
            const int64_t mid = (lo_r + hi_r) >> 1;
            if (mid * nb - mid * (mid - 1) / 2 <= item) lo_r = mid;
            else hi_r = mid;
        }
        const int64_t I = lo_r, J = I + (item - (I * nb - I * (I - 1) / 2));
        bool far = false;
        if (box && I / kPer != J / kPer) {
            const float *bi = box + 6 * (I / kPer), *bj = box + 6 * (J / kPer);
            float d2 = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float g = fmaxf(fmaxf(bj[c] - bi[3 + c], bi[c] - bj[3 + c]), 0.f);
                d2 = fmaf(g, g, d2);
            }
            far = d2 > far2;  // the same in every thread
        }
        if (far) dfsym_item<WALL, NT, true>(sD, sRev, hi, lo, f, n, I, J, k, u, scale);
        else dfsym_item<WALL, NT, false>(sD, sRev, hi, lo, f, n, I, J, k, u, scale);
    }
}

// u_i = scale * sum_s partial[s][i]  (fixed order)
__global__ void reduce_partials_kernel(const double *__restrict__ partial, int64_t n, int S,
                                       double scale, double *__restrict__ u)
{
    const int64_t m = 3 * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc += partial[s * m + e];
        u[e] = scale * acc;
    }
}

struct Plan {
    int n_tblocks = 0;
    int S = 1;
    int64_t chunk = 0;
    int64_t items = 0;
    int grid = 0;
};

// Split sources into S chunks so that the items fill whole waves of the
// resident grid as evenly as possible, with chunks of at least two tiles.
Plan make_plan(int64_t n, int targets_per_cta, int resident, int64_t s_cap = 64, int tile = kNT,
               int64_t min_chunk = 2 * kNT, int64_t n_src = -1)
{
    // n targets; n_src sources (the same blobs unless given)
    const int64_t ns = n_src < 0 ? n : n_src;
    Plan p;
    p.n_tblocks = (int)ceil_div(n, targets_per_cta);
    const int64_t max_s = std::max<int64_t>(1, std::min<int64_t>(s_cap, ceil_div(ns, min_chunk)));
    double best = -1.0;
    for (int64_t s = 1; s <= max_s; ++s) {
        const int64_t chunk = ceil_div(ceil_div(ns, s), tile) * tile;
        const int64_t s_eff = ceil_div(ns, chunk);
        const int64_t items = (int64_t)p.n_tblocks * s_eff;
        const int64_t waves = ceil_div(items, resident);
        double eff = (double)items / (double)(waves * resident);
        // a small preference for fewer chunks (less partial traffic)
        eff -= 1e-3 * (double)s_eff / 64.0;
        if (items < resident) eff *= (double)items / resident;
        if (eff > best + 1e-9) {
            best = eff;
            p.S = (int)s_eff;
            p.chunk = chunk;
        }
    }
    p.items = (int64_t)p.n_tblocks * p.S;
    p.grid = (int)std::min<int64_t>(p.items, resident);
    return p;
}

template <typename K>
int resident_ctas(mb_context *ctx, K kernel, int threads = kNT)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess ||
        occ < 1)
        occ = 1;
    return occ * ctx->sm_count;
}

constexpr int kTPT = MB_PAIR_TPT;  // targets per thread

}  // namespace

// ---------------------------------------------------------------------------
// FP32 variants and their autotuner.
//   0: scalar kernel, kTPT targets per thread
//   1: packed f32x2 kernel, 2 targets per thread
//   2: packed f32x2 kernel, 4 targets per thread
constexpr int kF32Variants = 5;
constexpr int kSmallNT = 32;        // CTA size of the small-problem kernels
constexpr int64_t kSmallN = 8192;   // below this the FP64 and double-float paths use them
constexpr int64_t kDfxMaxN = 1024;  // up to this the double-float product is forward only
constexpr int kSmallF64Chunk = 8;   // smallest source chunk of the small FP64 kernel

int f32_targets_per_cta(int v)
{
    return v == 0 ? kNT * kTPT : (v == 2 ? 4 * kNT : (v == 4 ? 2 * kSmallNT : 2 * kNT));
}

template <bool WALL>
int f32_resident(mb_context *ctx, int v)
{
    if (v == 0) return resident_ctas(ctx, pair_f32_kernel<WALL, kTPT>);
    if (v == 1) return resident_ctas(ctx, pair_f32x2_kernel<WALL, 1>);
    if (v == 3) return resident_ctas(ctx, pair_sym_kernel<WALL>);
    if (v == 4) return resident_ctas(ctx, pair_f32x2_kernel<WALL, 1, kSmallNT>, kSmallNT);
    return resident_ctas(ctx, pair_f32x2_kernel<WALL, 2>);
}

template <bool WALL>
void f32_launch(int v, const Plan &p, cudaStream_t s, const float4 *hi, const float4 *lo,
                const double *f, int64_t n, double a, double *out, double scale, int direct)
{
    if (v == 0) {
        pair_f32_kernel<WALL, kTPT><<<p.grid, kNT, 0, s>>>(
            hi, lo, f, n, p.chunk, p.n_tblocks, p.items, PairConsts<float>::make(a), out, scale,
            direct);
    } else if (v == 1) {
        pair_f32x2_kernel<WALL, 1><<<p.grid, kNT, 0, s>>>(
            hi, lo, f, n, p.chunk, p.n_tblocks, p.items, PairConsts2::make(a), out, scale, direct);
    } else if (v == 4) {
        pair_f32x2_kernel<WALL, 1, kSmallNT><<<p.grid, kSmallNT, 0, s>>>(
            hi, lo, f, n, p.chunk, p.n_tblocks, p.items, PairConsts2::make(a), out, scale, direct);
    } else {
        pair_f32x2_kernel<WALL, 2><<<p.grid, kNT, 0, s>>>(
            hi, lo, f, n, p.chunk, p.n_tblocks, p.items, PairConsts2::make(a), out, scale, direct);
    }
}

// ---------------------------------------------------------------------------
// Spatial order for the symmetric FP32 kernel (N >= kSortMinN).  The blobs are
// sorted by cell of a grid over their bounding box, cells in Morton order
// (kSortBits bits, dealt to the axes in proportion to their extents), by a
// counting sort; the kernel's blocks of 2 kNT consecutive sorted blobs are
// then compact, and the block pairs far apart take the FAR instance of the
// pair item.  Each matvec gathers f into the sorted order and scatters u back.
// The sort is stable (the blobs of a cell keep their index order), so the
// order, and with it the FP32 rounding of every pair sum, is the same on
// every call: a tile of consecutive blobs per CTA counts its keys in shared
// memory, the counts are scanned over tiles and buckets, and one warp per
// tile deals its blobs out in index order.  The grid has about N / 8 cells
// (2^10 .. 2^kSortBits): blocks of 512 blobs span a few dozen cells, and the
// per-tile count tables stay small.
constexpr int64_t kSortMinN = 16384;
constexpr int kSortBits = 15;         // most cell bits
constexpr int kSortKeysSmem = 16384;  // keys staged per round of the scatter

int sort_bits(int64_t n)
{
    int b = 10;  // at least 1,024 buckets (sort_scan_kernel's granule)
    while (b < kSortBits && ((int64_t)8 << b) < n) ++b;
    return b;
}

// The grid from the bounding box (ordered integers, as pack_hilo_kernel's
// partials): bits per axis by repeatedly halving the longest cell side, and
// the far distance, separations beyond 2^18 ulp of the largest coordinate.
__device__ void sort_grid_from_box(const unsigned *box, int nbits, SortGrid &g)
{
    float lo[3], ext[3], big = 0.f;
    for (int c = 0; c < 3; ++c) {
        lo[c] = order_float(box[c]);
        const float hi = order_float(box[3 + c]);
        ext[c] = fmaxf(hi - lo[c], 1e-30f);
        big = fmaxf(big, fmaxf(fabsf(lo[c]), fabsf(hi)));
    }
    int bits[3] = {0, 0, 0};
    for (int t = 0; t < nbits; ++t) {
        int a = 0;
        float best = -1.f;
        for (int c = 0; c < 3; ++c) {
            const float side = ldexpf(ext[c], -bits[c]);
            if (side > best) { best = side; a = c; }
        }
        ++bits[a];
    }
    for (int c = 0; c < 3; ++c) {
        g.lo[c] = lo[c];
        g.inv_h[c] = ldexpf(1.f, bits[c]) / ext[c];
        g.bits[c] = bits[c];
    }
    const float d = ldexpf(big, -23 + 18);
    g.far2 = d * d;
}

__device__ __forceinline__ unsigned sort_key(float4 h, const SortGrid &g)
{
    int q[3];
    const float x[3] = {h.x, h.y, h.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int top = (1 << g.bits[c]) - 1;
        q[c] = min(max((int)((x[c] - g.lo[c]) * g.inv_h[c]), 0), top);
    }
    unsigned key = 0;
    for (int l = kSortBits - 1; l >= 0; --l)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (g.bits[c] > l) key = (key << 1) | ((q[c] >> l) & 1);
    return key;
}

// tile b = blobs b T .. min(n, (b + 1) T) - 1: keys, and their counts per bucket
// (B = 2^nbits) in row b of H.  Every CTA first reduces the nparts
// bounding-box partials and forms the grid (CTA 0 also stores it for the
// pair kernel).
__global__ void __launch_bounds__(1024) sort_hist_kernel(const float4 *__restrict__ hi, int64_t n,
                                                         int64_t T, const unsigned *__restrict__ part,
                                                         int nparts, int nbits,
                                                         SortGrid *__restrict__ grid,
                                                         unsigned *__restrict__ key,
                                                         int *__restrict__ H)
{
    extern __shared__ int hist[];
    __shared__ unsigned red[6 * 32], box[6];
    __shared__ SortGrid gs;
    const int B = 1 << nbits;
    unsigned v[6] = {~0u, ~0u, ~0u, 0u, 0u, 0u};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < 6; ++c)
            v[c] = c < 3 ? min(v[c], part[6 * b + c]) : max(v[c], part[6 * b + c]);
    minmax_block(v, red, box);
    if (threadIdx.x == 0) {
        sort_grid_from_box(box, nbits, gs);
        if (blockIdx.x == 0) *grid = gs;
    }
    for (int c = threadIdx.x; c < B; c += blockDim.x) hist[c] = 0;
    __syncthreads();
    const SortGrid g = gs;
    const int64_t i0 = blockIdx.x * T, i1 = min(n, i0 + T);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const unsigned k = sort_key(hi[i], g);
        key[i] = k;
        atomicAdd(hist + k, 1);
    }
    __syncthreads();
    int *row = H + blockIdx.x * (int64_t)B;
    for (int c = threadIdx.x; c < B; c += blockDim.x) row[c] = hist[c];
}

// per bucket (one thread each): rows 0..tiles-1 of H become the exclusive
// prefix over tiles, row `tiles` the bucket's total (the loads of up to 32
// tiles in flight at once)
__global__ void __launch_bounds__(256) sort_tile_scan_kernel(int *__restrict__ H, int tiles, int B)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    int run = 0;
    for (int b0 = 0; b0 < tiles; b0 += 32) {
        int t[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) t[u] = b0 + u < tiles ? H[(b0 + u) * (int64_t)B + c] : 0;
#pragma unroll
        for (int u = 0; u < 32; ++u)
            if (b0 + u < tiles) {
                H[(b0 + u) * (int64_t)B + c] = run;
                run += t[u];
            }
    }
    H[tiles * (int64_t)B + c] = run;
}

// exclusive scan of the B counters in one CTA of 1024 threads: the counters
// staged in shared memory (coalesced; one pad word per 32 so that thread t's
// run of B / 1024 consecutive counters is free of bank conflicts), a
// sequential sum per thread, a scan of the 1024 sums, the prefixes written
// back through shared memory
__device__ __forceinline__ int scan_pad(int e) { return e + (e >> 5); }

__global__ void __launch_bounds__(1024) sort_scan_kernel(int *__restrict__ count, int B)
{
    extern __shared__ int sc[];
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = B >> 10;  // B is a power of two >= 1024
    for (int e = threadIdx.x; e < B; e += 1024) sc[scan_pad(e)] = count[e];
    __syncthreads();
    const int e0 = threadIdx.x * per;
    int tot = 0;
    for (int k = 0; k < per; ++k) tot += sc[scan_pad(e0 + k)];
    int x = tot;  // inclusive scan of the per-thread sums
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int y = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        wsum[lane] = y;
    }
    __syncthreads();
    int run = (warp > 0 ? wsum[warp - 1] : 0) + x - tot;
    for (int k = 0; k < per; ++k) {
        const int v = sc[scan_pad(e0 + k)];
        sc[scan_pad(e0 + k)] = run;
        run += v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < B; e += 1024) count[e] = sc[scan_pad(e)];
}

// perm[position] = blob.  Tile b's first position in bucket k is start[k] +
// H[b][k]; warp 0 takes the tile's keys 32 at a time in index order, ranks
// equal keys among its lanes (match), and advances the bucket's offset in
// shared memory once per group.
__global__ void __launch_bounds__(1024) sort_scatter_kernel(const unsigned *__restrict__ key,
                                                            int64_t n, int64_t T,
                                                            const int *__restrict__ H, int tiles,
                                                            int B, int *__restrict__ perm)
{
    extern __shared__ int off[];
    unsigned *sk = (unsigned *)(off + B);
    const int *row = H + blockIdx.x * (int64_t)B;
    const int *start = H + tiles * (int64_t)B;
    for (int c = threadIdx.x; c < B; c += blockDim.x) off[c] = start[c] + row[c];
    const int64_t i0 = blockIdx.x * T, i1 = min(n, i0 + T);
    for (int64_t c0 = i0; c0 < i1; c0 += kSortKeysSmem) {
        const int m = (int)min((int64_t)kSortKeysSmem, i1 - c0);
        __syncthreads();  // offsets written; warp 0 done with the previous round's keys
        for (int e = threadIdx.x; e < m; e += blockDim.x) sk[e] = key[c0 + e];
        __syncthreads();
        if (threadIdx.x < 32) {
            // the leader of each group of equal keys reads and advances the
            // bucket's offset and hands the base to its group; the next
            // chunk's key is loaded one round ahead
            const unsigned lane = threadIdx.x;
            unsigned k_next = (int)lane < m ? sk[lane] : 0xffffffffu;  // no bucket has this key
            for (int e0 = 0; e0 < m; e0 += 32) {
                const int e = e0 + (int)lane;
                const bool ok = e < m;
                const unsigned k = k_next;
                k_next = e + 32 < m ? sk[e + 32] : 0xffffffffu;
                const unsigned same = __match_any_sync(0xffffffffu, k);
                const int leader = __ffs(same) - 1;
                int base = 0;
                if (ok && (int)lane == leader) {
                    base = off[k];
                    off[k] = base + __popc(same);
                }
                base = __shfl_sync(0xffffffffu, base, leader);
                if (ok) perm[base + __popc(same & ((1u << lane) - 1u))] = (int)(c0 + e);
                __syncwarp();  // this round's offsets before the next round's reads
            }
        }
    }
}

// Block b of the kernel (sorted positions b * 2 kNT .. + 2 kNT - 1), one CTA
// each: the packed positions in the sorted order, and the block's bounding
// box (min x, y, z, max x, y, z).
__global__ void __launch_bounds__(256) sort_pack_box_kernel(const int *__restrict__ perm, int64_t n,
                                                            const float4 *__restrict__ hi,
                                                            const float4 *__restrict__ lo,
                                                            float4 *__restrict__ shi,
                                                            float4 *__restrict__ slo,
                                                            float *__restrict__ box)
{
    __shared__ float red[32][6];
    const int64_t b = blockIdx.x;
    float v[6] = {3e38f, 3e38f, 3e38f, -3e38f, -3e38f, -3e38f};
    for (int64_t i = b * 2 * kNT + threadIdx.x; i < n && i < (b + 1) * 2 * kNT; i += blockDim.x) {
        const int j = perm[i];
        const float4 h = hi[j];
        shi[i] = h;
        slo[i] = lo[j];
        v[0] = fminf(v[0], h.x); v[1] = fminf(v[1], h.y); v[2] = fminf(v[2], h.z);
        v[3] = fmaxf(v[3], h.x); v[4] = fmaxf(v[4], h.y); v[5] = fmaxf(v[5], h.z);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float t = __shfl_xor_sync(0xffffffffu, v[c], o);
            v[c] = c < 3 ? fminf(v[c], t) : fmaxf(v[c], t);
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) red[threadIdx.x >> 5][c] = v[c];
    __syncthreads();
    if (threadIdx.x < 6) {
        float r = red[0][threadIdx.x];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            r = threadIdx.x < 3 ? fminf(r, red[w][threadIdx.x]) : fmaxf(r, red[w][threadIdx.x]);
        box[6 * b + threadIdx.x] = r;
    }
}

// f into the sorted order, and the sorted velocities zeroed (the pair
// kernel adds into them)
__global__ void __launch_bounds__(256) sort_gather_kernel(const int *__restrict__ perm, int64_t n,
                                                          const double *__restrict__ f,
                                                          double *__restrict__ fs,
                                                          double *__restrict__ us)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = perm[i];
        fs[3 * i] = f[3 * j];
        fs[3 * i + 1] = f[3 * j + 1];
        fs[3 * i + 2] = f[3 * j + 2];
        us[3 * i] = 0.0;
        us[3 * i + 1] = 0.0;
        us[3 * i + 2] = 0.0;
    }
}

__global__ void __launch_bounds__(256) sort_scatter_u_kernel(const int *__restrict__ perm,
                                                             int64_t n,
                                                             const double *__restrict__ us,
                                                             double *__restrict__ u)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = perm[i];
        u[3 * j] = us[3 * i];
        u[3 * j + 1] = us[3 * i + 1];
        u[3 * j + 2] = us[3 * i + 2];
    }
}

// The order of the packed positions, for N >= kSortMinN: pack_hilo_kernel
// has left nparts bounding-box partials in the sort_grid buffer (after the
// SortGrid).
mb_status sort_positions(mb_context *ctx, int64_t n, int nparts, cudaStream_t s)
{
    const int64_t nb = ceil_div(n, 2 * kNT);
    // tiles of at least 1,024 blobs, at most one per SM
    const int tiles = (int)std::min<int64_t>(ceil_div(n, 1024), ctx->sm_count);
    const int64_t T = ceil_div(n, tiles);
    MB_TRY(ensure(ctx, ctx->sort_perm, sizeof(int) * (size_t)n, "spatial order"));
    MB_TRY(ensure(ctx, ctx->sort_key, sizeof(unsigned) * (size_t)n, "spatial order"));
    const int nbits = sort_bits(n), B = 1 << nbits;
    const size_t hist_smem = sizeof(int) * (size_t)B;
    const size_t scan_smem = sizeof(int) * (size_t)(B + B / 32);
    const size_t scatter_smem = hist_smem + sizeof(unsigned) * kSortKeysSmem;
    MB_TRY(ensure(ctx, ctx->sort_count, hist_smem * (size_t)(tiles + 1), "spatial order"));
    MB_TRY(ensure(ctx, ctx->sort_hi, sizeof(float4) * (size_t)n, "spatial order"));
    MB_TRY(ensure(ctx, ctx->sort_lo, sizeof(float4) * (size_t)n, "spatial order"));
    MB_TRY(ensure(ctx, ctx->sort_box, sizeof(float) * 6 * (size_t)nb, "spatial order"));
    MB_CUDA_TRY(ctx, cudaFuncSetAttribute(sort_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)hist_smem));
    MB_CUDA_TRY(ctx, cudaFuncSetAttribute(sort_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)scan_smem));
    MB_CUDA_TRY(ctx, cudaFuncSetAttribute(sort_scatter_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)scatter_smem));
    SortGrid *grid = (SortGrid *)ctx->sort_grid.ptr;
    const unsigned *part = (const unsigned *)((char *)ctx->sort_grid.ptr + sizeof(SortGrid));
    const float4 *hi = (const float4 *)ctx->pos_hi.ptr, *lo = (const float4 *)ctx->pos_lo.ptr;
    int *H = (int *)ctx->sort_count.ptr;
    unsigned *key = (unsigned *)ctx->sort_key.ptr;
    sort_hist_kernel<<<tiles, 1024, hist_smem, s>>>(hi, n, T, part, nparts, nbits, grid, key, H);
    sort_tile_scan_kernel<<<(B + 255) / 256, 256, 0, s>>>(H, tiles, B);
    sort_scan_kernel<<<1, 1024, scan_smem, s>>>(H + tiles * (int64_t)B, B);
    sort_scatter_kernel<<<tiles, 1024, scatter_smem, s>>>(key, n, T, H, tiles, B,
                                                          (int *)ctx->sort_perm.ptr);
    sort_pack_box_kernel<<<(int)nb, 256, 0, s>>>((const int *)ctx->sort_perm.ptr, n, hi, lo,
                                                 (float4 *)ctx->sort_hi.ptr,
                                                 (float4 *)ctx->sort_lo.ptr,
                                                 (float *)ctx->sort_box.ptr);
    count_launch(5);
    MB_CUDA_TRY(ctx, cudaGetLastError());
    ctx->sorted_n = n;
    return MB_OK;
}

// One FP32 matvec with variant v (pair kernel + chunk reduction).
mb_status f32_run(mb_context *ctx, int v, const double *f, int64_t n, double a, int wall,
                  double scale, double *u, cudaStream_t s, bool profile,
                  MatvecPartials *defer = nullptr)
{
    const int res = wall ? f32_resident<true>(ctx, v) : f32_resident<false>(ctx, v);
    if (v == 4) {
        // small problems: 64-target blocks, source chunks of 16 or more (half a
        // tile: one warp per CTA walks fewer sources, more CTAs share the work)
        const Plan p = make_plan(n, f32_targets_per_cta(4), res, 1024, kSmallNT / 2, kSmallNT / 2);
        double *out = u;
        const int direct = p.S == 1;
        if (!direct) {
            MB_TRY(ensure(ctx, ctx->partial, sizeof(double) * 3 * (size_t)n * p.S, "matvec partials"));
            out = (double *)ctx->partial.ptr;
        }
        auto *ev = profile ? profile_begin(ctx, s) : nullptr;
        const float4 *hi = (const float4 *)ctx->pos_hi.ptr;
        const float4 *lo = (const float4 *)ctx->pos_lo.ptr;
        if (wall)
            f32_launch<true>(4, p, s, hi, lo, f, n, a, out, scale, direct);
        else
            f32_launch<false>(4, p, s, hi, lo, f, n, a, out, scale, direct);
        profile_end(ev, s);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
        if (!direct) {
            if (defer) {
                *defer = MatvecPartials{out, p.S, scale};
                return MB_OK;
            }
            const int grid = (int)std::min<int64_t>(ceil_div(3 * n, 256), 8 * (int64_t)ctx->sm_count);
            reduce_partials_kernel<<<grid, 256, 0, s>>>(out, n, p.S, scale, u);
            count_launch();
            MB_CUDA_TRY(ctx, cudaGetLastError());
        }
        return MB_OK;
    }
    if (v == 3) {
        // symmetric: zero u, then one launch over the block-pair triangle; in
        // the spatial order when the packing made one (f gathered, u
        // scattered back)
        const int64_t nb = ceil_div(n, 2 * kNT);
        const int64_t items = nb * (nb + 1) / 2;
        const int grid = (int)std::min<int64_t>(items, res);
        const bool sorted = ctx->sorted_n == n;
        const float4 *hi = (const float4 *)(sorted ? ctx->sort_hi.ptr : ctx->pos_hi.ptr);
        const float4 *lo = (const float4 *)(sorted ? ctx->sort_lo.ptr : ctx->pos_lo.ptr);
        const float *box = sorted ? (const float *)ctx->sort_box.ptr : nullptr;
        const SortGrid *sg = sorted ? (const SortGrid *)ctx->sort_grid.ptr : nullptr;
        const double *fk = f;
        double *uk = u;
        const int gv = (int)std::min<int64_t>(ceil_div(n, 256), 8 * (int64_t)ctx->sm_count);
        if (sorted) {
            MB_TRY(ensure(ctx, ctx->sort_f, sizeof(double) * 3 * (size_t)n, "sorted forces"));
            MB_TRY(ensure(ctx, ctx->sort_u, sizeof(double) * 3 * (size_t)n, "sorted velocities"));
            sort_gather_kernel<<<gv, 256, 0, s>>>((const int *)ctx->sort_perm.ptr, n, f,
                                                  (double *)ctx->sort_f.ptr,
                                                  (double *)ctx->sort_u.ptr);
            count_launch();
            fk = (const double *)ctx->sort_f.ptr;
            uk = (double *)ctx->sort_u.ptr;
        } else {
            MB_CUDA_TRY(ctx, cudaMemsetAsync(uk, 0, sizeof(double) * 3 * (size_t)n, s));
        }
        auto *ev = profile ? profile_begin(ctx, s) : nullptr;
        const PairConsts2 k = PairConsts2::make(a);
        if (wall)
            pair_sym_kernel<true><<<grid, kNT, 0, s>>>(hi, lo, fk, n, nb, items, k, uk, scale, box, sg);
        else
            pair_sym_kernel<false><<<grid, kNT, 0, s>>>(hi, lo, fk, n, nb, items, k, uk, scale, box, sg);
        profile_end(ev, s);
        count_launch();
        if (sorted) {
            sort_scatter_u_kernel<<<gv, 256, 0, s>>>((const int *)ctx->sort_perm.ptr, n, uk, u);
            count_launch();
        }
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }
    const Plan p = make_plan(n, f32_targets_per_cta(v), res);
    double *out = u;
    const int direct = p.S == 1;
    if (!direct) {
        MB_TRY(ensure(ctx, ctx->partial, sizeof(double) * 3 * (size_t)n * p.S, "matvec partials"));
        out = (double *)ctx->partial.ptr;
    }
    auto *ev = profile ? profile_begin(ctx, s) : nullptr;
    const float4 *hi = (const float4 *)ctx->pos_hi.ptr;
    const float4 *lo = (const float4 *)ctx->pos_lo.ptr;
    if (wall)
        f32_launch<true>(v, p, s, hi, lo, f, n, a, out, scale, direct);
    else
        f32_launch<false>(v, p, s, hi, lo, f, n, a, out, scale, direct);
    profile_end(ev, s);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    if (!direct && defer) {
        *defer = MatvecPartials{out, p.S, scale};
        return MB_OK;
    }
    if (!direct) {
        const int grid = (int)std::min<int64_t>(ceil_div(3 * n, 256), 8 * (int64_t)ctx->sm_count);
        reduce_partials_kernel<<<grid, 256, 0, s>>>(out, n, p.S, scale, u);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
    }
    return MB_OK;
}

// Size class of a matvec for the autotuner: wall flag and half-octaves of N.
int tune_key(int64_t n, int wall)
{
    int b = 0;
    for (int64_t m = n; m > 1; m >>= 1) ++b;
    const int half = (n >= 3 * ((int64_t)1 << (b > 0 ? b - 1 : 0))) ? 1 : 0;
    return (2 * b + half) * 2 + (wall ? 1 : 0);
}

mb_status matvec_f32(mb_context *ctx, const double *f, int64_t n, double a, int wall,
                     double scale, double *u, cudaStream_t s, MatvecPartials *defer)
{
    int v = ctx->pair_variant;
    if (v < 0) {
        const int key = tune_key(n, wall);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            v = it->second;
        } else if (n < 4096) {
            v = 4;  // small: spread over many SMs in 64-target, 32-source items
            ctx->tuned[key] = v;
        } else {
            // time each variant once on this stream (each run is a full, valid matvec)
            float best = 1e30f;
            int best_v = 1;
            cudaEvent_t e0, e1;
            MB_CUDA_TRY(ctx, cudaEventCreate(&e0));
            MB_CUDA_TRY(ctx, cudaEventCreate(&e1));
            for (int c = 0; c < kF32Variants; ++c) {
                MB_CUDA_TRY(ctx, cudaEventRecord(e0, s));
                MB_TRY(f32_run(ctx, c, f, n, a, wall, scale, u, s, false));
                MB_CUDA_TRY(ctx, cudaEventRecord(e1, s));
                MB_CUDA_TRY(ctx, cudaEventSynchronize(e1));
                float ms = 0.f;
                MB_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; best_v = c; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ctx->tuned[key] = best_v;
            v = best_v;
        }
    }
    return f32_run(ctx, v, f, n, a, wall, scale, u, s, true, defer);
}

mb_status matvec_pack_positions(mb_context *ctx, const double *r, int64_t n, cudaStream_t s,
                                bool order)
{
    MB_TRY(ensure(ctx, ctx->pos_hi, sizeof(float4) * (size_t)n, "packed positions"));
    MB_TRY(ensure(ctx, ctx->pos_lo, sizeof(float4) * (size_t)n, "packed positions"));
    ctx->sorted_n = 0;
    const int grid = (int)std::min<int64_t>(ceil_div(n, 256), 8 * (int64_t)ctx->sm_count);
    const bool sort = order && n >= kSortMinN;
    if (sort) {
        MB_TRY(ensure(ctx, ctx->sort_grid, sizeof(SortGrid) + sizeof(unsigned) * 6 * (size_t)grid,
                      "spatial order"));
        pack_hilo_kernel<true><<<grid, 256, 0, s>>>(
            r, n, (float4 *)ctx->pos_hi.ptr, (float4 *)ctx->pos_lo.ptr,
            (unsigned *)((char *)ctx->sort_grid.ptr + sizeof(SortGrid)));
    } else {
        pack_hilo_kernel<false><<<grid, 256, 0, s>>>(r, n, (float4 *)ctx->pos_hi.ptr,
                                                     (float4 *)ctx->pos_lo.ptr, nullptr);
    }
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    if (sort) MB_TRY(sort_positions(ctx, n, grid, s));
    return MB_OK;
}

mb_status matvec_packed(mb_context *ctx, const double *r, const double *f, int64_t n, double a,
                        double eta, int wall, mb_precision prec, double *u, cudaStream_t s,
                        MatvecPartials *defer)
{
    const double scale = 1.0 / (6.0 * kPi * eta * a);
    if (defer) *defer = MatvecPartials{};
    if (prec == MB_FP32_KAHAN) return matvec_f32(ctx, f, n, a, wall, scale, u, s, defer);
    if (prec == MB_DF64) {
        // symmetric double-float kernel: zero u, one launch over the block-pair
        // triangle (32-blob blocks for small problems, so that they spread)
        const bool small = n < kSmallN;
        const int nt = small ? kSmallNT : kNT;
        const int res = small ? (wall ? resident_ctas(ctx, pair_df_kernel<true, kSmallNT>, kSmallNT)
                                      : resident_ctas(ctx, pair_df_kernel<false, kSmallNT>, kSmallNT))
                              : (wall ? resident_ctas(ctx, pair_df_kernel<true>)
                                      : resident_ctas(ctx, pair_df_kernel<false>));
        const int64_t nb = ceil_div(n, nt);
        const int64_t items = nb * (nb + 1) / 2;
        const int grid = (int)std::min<int64_t>(items, res);
        // in the spatial order when the packing made one (f gathered, u
        // scattered back): far block pairs take the cheaper FAR item
        const bool sorted = !small && ctx->sorted_n == n;
        const float4 *hi = (const float4 *)(sorted ? ctx->sort_hi.ptr : ctx->pos_hi.ptr);
        const float4 *lo = (const float4 *)(sorted ? ctx->sort_lo.ptr : ctx->pos_lo.ptr);
        const float *box = sorted ? (const float *)ctx->sort_box.ptr : nullptr;
        const float dfar = (float)(64.0 * a);
        const double *fk = f;
        double *uk = u;
        const int gv = (int)std::min<int64_t>(ceil_div(n, 256), 8 * (int64_t)ctx->sm_count);
        if (sorted) {
            MB_TRY(ensure(ctx, ctx->sort_f, sizeof(double) * 3 * (size_t)n, "sorted forces"));
            MB_TRY(ensure(ctx, ctx->sort_u, sizeof(double) * 3 * (size_t)n, "sorted velocities"));
            sort_gather_kernel<<<gv, 256, 0, s>>>((const int *)ctx->sort_perm.ptr, n, f,
                                                  (double *)ctx->sort_f.ptr,
                                                  (double *)ctx->sort_u.ptr);
            count_launch();
            fk = (const double *)ctx->sort_f.ptr;
            uk = (double *)ctx->sort_u.ptr;
        } else {
            MB_CUDA_TRY(ctx, cudaMemsetAsync(u, 0, sizeof(double) * 3 * (size_t)n, s));
        }
        auto *ev = profile_begin(ctx, s);
        const PairConsts<dfl> k = PairConsts<dfl>::make(a);
        if (n <= kDfxMaxN) {
            // the smallest problems: every ordered pair, many one-warp CTAs
            const int rx = wall ? resident_ctas(ctx, pair_dfx_kernel<true, kSmallNT>, kSmallNT)
                                : resident_ctas(ctx, pair_dfx_kernel<false, kSmallNT>, kSmallNT);
            const Plan px = make_plan(n, kSmallNT, rx, 1024, kSmallNT / 2, kSmallNT / 2);
            if (wall)
                pair_dfx_kernel<true, kSmallNT><<<px.grid, kSmallNT, 0, s>>>(hi, lo, fk, n, px.chunk,
                                                                   px.n_tblocks, px.items, k, uk,
                                                                   scale);
            else
                pair_dfx_kernel<false, kSmallNT><<<px.grid, kSmallNT, 0, s>>>(hi, lo, fk, n, px.chunk,
                                                                    px.n_tblocks, px.items, k, uk,
                                                                    scale);
        } else if (small && wall)
            pair_df_kernel<true, kSmallNT><<<grid, kSmallNT, 0, s>>>(hi, lo, fk, n, nb, items, k, uk,
                                                                    scale, nullptr, 0.f);
        else if (small)
            pair_df_kernel<false, kSmallNT><<<grid, kSmallNT, 0, s>>>(hi, lo, fk, n, nb, items, k,
                                                                     uk, scale, nullptr, 0.f);
        else if (wall)
            pair_df_kernel<true><<<grid, kNT, 0, s>>>(hi, lo, fk, n, nb, items, k, uk, scale, box,
                                                      dfar * dfar);
        else
            pair_df_kernel<false><<<grid, kNT, 0, s>>>(hi, lo, fk, n, nb, items, k, uk, scale, box,
                                                       dfar * dfar);
        profile_end(ev, s);
        count_launch();
        if (sorted) {
            sort_scatter_u_kernel<<<gv, 256, 0, s>>>((const int *)ctx->sort_perm.ptr, n, uk, u);
            count_launch();
        }
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }
    const bool small = n < kSmallN;
    if (!small) {
        // symmetric FP64 kernel: zero u, one launch over the block-pair triangle
        const int res = wall ? resident_ctas(ctx, pair_f64sym_kernel<true>)
                             : resident_ctas(ctx, pair_f64sym_kernel<false>);
        const int64_t nb = ceil_div(n, kNT);
        const int64_t items = nb * (nb + 1) / 2;
        const int grid = (int)std::min<int64_t>(items, res);
        MB_CUDA_TRY(ctx, cudaMemsetAsync(u, 0, sizeof(double) * 3 * (size_t)n, s));
        auto *ev = profile_begin(ctx, s);
        const PairConsts<double> k = PairConsts<double>::make(a);
        if (wall)
            pair_f64sym_kernel<true><<<grid, kNT, 0, s>>>(r, f, n, nb, items, k, u, scale);
        else
            pair_f64sym_kernel<false><<<grid, kNT, 0, s>>>(r, f, n, nb, items, k, u, scale);
        profile_end(ev, s);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
        return MB_OK;
    }
    Plan p;
    if (small) {
        const int res = wall ? resident_ctas(ctx, pair_f64_kernel<true, kSmallNT>, kSmallNT)
                             : resident_ctas(ctx, pair_f64_kernel<false, kSmallNT>, kSmallNT);
        // source chunks down to 8 blobs: several one-warp CTAs per SM, since
        // a single warp leaves the FP64 pipe mostly idle
        p = make_plan(n, kSmallNT, res, 1024, kSmallF64Chunk, kSmallF64Chunk);
    } else {
        const int res = wall ? resident_ctas(ctx, pair_f64_kernel<true>)
                             : resident_ctas(ctx, pair_f64_kernel<false>);
        p = make_plan(n, kNT, res);
    }
    double *out = u;
    const int direct = p.S == 1;
    if (!direct) {
        MB_TRY(ensure(ctx, ctx->partial, sizeof(double) * 3 * (size_t)n * p.S, "matvec partials"));
        out = (double *)ctx->partial.ptr;
    }
    auto *ev = profile_begin(ctx, s);
    const PairConsts<double> k = PairConsts<double>::make(a);
    if (small && wall)
        pair_f64_kernel<true, kSmallNT><<<p.grid, kSmallNT, 0, s>>>(r, f, n, p.chunk, p.n_tblocks,
                                                                   p.items, k, out, scale, direct);
    else if (small)
        pair_f64_kernel<false, kSmallNT><<<p.grid, kSmallNT, 0, s>>>(r, f, n, p.chunk, p.n_tblocks,
                                                                    p.items, k, out, scale, direct);
    else if (wall)
        pair_f64_kernel<true><<<p.grid, kNT, 0, s>>>(r, f, n, p.chunk, p.n_tblocks, p.items, k, out,
                                                     scale, direct);
    else
        pair_f64_kernel<false><<<p.grid, kNT, 0, s>>>(r, f, n, p.chunk, p.n_tblocks, p.items, k,
                                                      out, scale, direct);
    profile_end(ev, s);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    if (!direct && defer) {
        *defer = MatvecPartials{out, p.S, scale};
        return MB_OK;
    }
    if (!direct) {
        const int grid = (int)std::min<int64_t>(ceil_div(3 * n, 256), 8 * (int64_t)ctx->sm_count);
        reduce_partials_kernel<<<grid, 256, 0, s>>>(out, n, p.S, scale, u);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
    }
    return MB_OK;
}

mb_status matvec_device(mb_context *ctx, const double *r, const double *f, int64_t n, double a,
                        double eta, int wall, mb_precision prec, double *u, cudaStream_t s)
{
    if (prec != MB_FP64) MB_TRY(matvec_pack_positions(ctx, r, n, s));
    return matvec_packed(ctx, r, f, n, a, eta, wall, prec, u, s);
}

mb_status matvec_eval(mb_context *ctx, const double *x, int64_t nt, const double *r,
                      const double *f, int64_t ns, double a, double eta, int wall,
                      mb_precision prec, double *u, cudaStream_t s)
{
    const double scale = 1.0 / (6.0 * kPi * eta * a);
    if (prec == MB_FP64) {
        const int res = wall ? resident_ctas(ctx, eval_f64_kernel<true>)
                             : resident_ctas(ctx, eval_f64_kernel<false>);
        const Plan p = make_plan(nt, kNT, res, 64, kNT, 2 * kNT, ns);
        double *out = u;
        const int direct = p.S == 1;
        if (!direct) {
            MB_TRY(ensure(ctx, ctx->partial, sizeof(double) * 3 * (size_t)nt * p.S, "eval partials"));
            out = (double *)ctx->partial.ptr;
        }
        const PairConsts<double> k = PairConsts<double>::make(a);
        if (wall)
            eval_f64_kernel<true><<<p.grid, kNT, 0, s>>>(x, nt, r, f, ns, p.chunk, p.n_tblocks,
                                                         p.items, k, out, scale, direct);
        else
            eval_f64_kernel<false><<<p.grid, kNT, 0, s>>>(x, nt, r, f, ns, p.chunk, p.n_tblocks,
                                                          p.items, k, out, scale, direct);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
        if (!direct) {
            const int grid = (int)std::min<int64_t>(ceil_div(3 * nt, 256), 8 * (int64_t)ctx->sm_count);
            reduce_partials_kernel<<<grid, 256, 0, s>>>(out, nt, p.S, scale, u);
            count_launch();
            MB_CUDA_TRY(ctx, cudaGetLastError());
        }
        return MB_OK;
    }
    if (prec != MB_FP32_KAHAN)
        return set_err(ctx, MB_EINVAL, "flow evaluation supports MB_FP32_KAHAN and MB_FP64");
    // sources packed into the context's position buffers, targets into the eval ones
    MB_TRY(matvec_pack_positions(ctx, r, ns, s, false));
    MB_TRY(ensure(ctx, ctx->eval_hi, sizeof(float4) * (size_t)nt, "packed targets"));
    MB_TRY(ensure(ctx, ctx->eval_lo, sizeof(float4) * (size_t)nt, "packed targets"));
    {
        const int grid = (int)std::min<int64_t>(ceil_div(nt, 256), 8 * (int64_t)ctx->sm_count);
        pack_hilo_kernel<false><<<grid, 256, 0, s>>>(x, nt, (float4 *)ctx->eval_hi.ptr,
                                                     (float4 *)ctx->eval_lo.ptr, nullptr);
        count_launch();
    }
    const int res = wall ? resident_ctas(ctx, eval_f32x2_kernel<true>)
                         : resident_ctas(ctx, eval_f32x2_kernel<false>);
    const Plan p = make_plan(nt, 2 * kNT, res, 64, kNT, 2 * kNT, ns);
    double *out = u;
    const int direct = p.S == 1;
    if (!direct) {
        MB_TRY(ensure(ctx, ctx->partial, sizeof(double) * 3 * (size_t)nt * p.S, "eval partials"));
        out = (double *)ctx->partial.ptr;
    }
    const PairConsts2 k = PairConsts2::make(a);
    const float4 *thi = (const float4 *)ctx->eval_hi.ptr, *tlo = (const float4 *)ctx->eval_lo.ptr;
    const float4 *hi = (const float4 *)ctx->pos_hi.ptr, *lo = (const float4 *)ctx->pos_lo.ptr;
    if (wall)
        eval_f32x2_kernel<true><<<p.grid, kNT, 0, s>>>(thi, tlo, nt, hi, lo, f, ns, p.chunk,
                                                       p.n_tblocks, p.items, k, out, scale, direct);
    else
        eval_f32x2_kernel<false><<<p.grid, kNT, 0, s>>>(thi, tlo, nt, hi, lo, f, ns, p.chunk,
                                                        p.n_tblocks, p.items, k, out, scale, direct);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    if (!direct) {
        const int grid = (int)std::min<int64_t>(ceil_div(3 * nt, 256), 8 * (int64_t)ctx->sm_count);
        reduce_partials_kernel<<<grid, 256, 0, s>>>(out, nt, p.S, scale, u);
        count_launch();
        MB_CUDA_TRY(ctx, cudaGetLastError());
    }
    return MB_OK;
}

mb_status render_flow(mb_context *ctx, const double *x, int64_t nt, const double *r,
                      const double *lam, int64_t n, const double *off, int n_sub, double a_sub,
                      double eta, int wall, mb_precision prec, double *v, cudaStream_t s)
{
    const int64_t ns = n * (int64_t)n_sub;
    MB_TRY(ensure(ctx, ctx->render_r, sizeof(double) * 3 * (size_t)ns, "refined blobs"));
    MB_TRY(ensure(ctx, ctx->render_f, sizeof(double) * 3 * (size_t)ns, "refined blob forces"));
    const int grid = (int)std::min<int64_t>(ceil_div(ns, 256), 8 * (int64_t)ctx->sm_count);
    refine_blobs_kernel<<<grid, 256, 0, s>>>(r, lam, n, off, n_sub, (double *)ctx->render_r.ptr,
                                             (double *)ctx->render_f.ptr);
    count_launch();
    MB_CUDA_TRY(ctx, cudaGetLastError());
    return matvec_eval(ctx, x, nt, (const double *)ctx->render_r.ptr,
                       (const double *)ctx->render_f.ptr, ns, a_sub, eta, wall, prec, v, s);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP32 matvec (mb_mobility_matvec_noalloc).
//
// For callers that must not allocate device memory: host applications whose
// framework owns the whole device-memory budget (a caching allocator has
// reserved it, so a cudaMalloc would fail or fragment it) and code on
// latency-critical paths that cannot take cudaMalloc's implicit device
// synchronisation.  The scratch that mb_mobility_matvec keeps in its context
// (packed hi/lo positions and per-chunk partial sums) lives here in one
// file-scope device array instead, sized for MB_NOALLOC_MAX_BLOBS blobs and at
// most kNoallocMaxChunks source chunks.  Every GPU that loads the library
// holds the array until the process exits.  All calls share it: calls whose
// work overlaps on the GPU race on it.  Each call writes every element it
// later reads, so nothing needs clearing between calls.
namespace {

constexpr int64_t kNoallocMaxBlobs = MB_NOALLOC_MAX_BLOBS;
constexpr int kNoallocMaxChunks = 8;
constexpr size_t kNoallocPosBytes = sizeof(float4) * kNoallocMaxBlobs;
constexpr size_t kNoallocBytes =
    2 * kNoallocPosBytes + sizeof(double) * 3 * kNoallocMaxChunks * kNoallocMaxBlobs;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

struct NoallocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int resident_wall = 0, resident_free = 0;
};
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[kNoallocMaxDevices];

// First call on a device: look up the array's device address (host code may
// not use the symbol itself) and the resident-grid sizes.  No allocation.
mb_status noalloc_setup(int dev, NoallocDevice **out)
{
    if (dev < 0 || dev >= kNoallocMaxDevices) return MB_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            set_thread_err("cudaGetSymbolAddress of the allocation-free scratch failed");
            return MB_ECUDA;
        }
        int sms = 0, occ_w = 0, occ_f = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_w, pair_f32_kernel<true, kTPT>,
                                                          kNT, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, pair_f32_kernel<false, kTPT>,
                                                          kNT, 0) != cudaSuccess) {
            cudaGetLastError();
            set_thread_err("device query failed in the allocation-free matvec set-up");
            return MB_ECUDA;
        }
        d.scratch = (unsigned char *)ptr;
        d.resident_wall = std::max(1, occ_w) * sms;
        d.resident_free = std::max(1, occ_f) * sms;
        d.ready = true;
    }
    *out = &d;
    return MB_OK;
}

// Device memory of device `dev` (the one whose scratch array the call uses),
// or managed memory.  Memory of another GPU would reach the kernel as a peer
// pointer, so it is refused on the host instead.
bool on_device(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice && at.device == dev) ||
           at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace mb

extern "C" mb_status mb_mobility_matvec_noalloc(const double *r, const double *f, int64_t n,
                                                double a, double eta, int wall, double *u,
                                                void *stream)
{
    using namespace mb;
    set_thread_err("");
    if (n < 0 || n > kNoallocMaxBlobs) {
        set_thread_err("N must be in [0, MB_NOALLOC_MAX_BLOBS]");
        return MB_EINVAL;
    }
    if (!(a > 0.0) || !(eta > 0.0)) {
        set_thread_err("a and eta must be positive");
        return MB_EINVAL;
    }
    if (n == 0) return MB_OK;
    if (!r || !f || !u) {
        set_thread_err("r, f and u must be device pointers");
        return MB_EINVAL;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_thread_err("cudaGetDevice failed");
        return MB_ECUDA;
    }
    if (!on_device(r, dev) || !on_device(f, dev) || !on_device(u, dev)) {
        set_thread_err("r, f and u must be device pointers on the current device");
        return MB_EINVAL;
    }
    NoallocDevice *d = nullptr;
    mb_status st = noalloc_setup(dev, &d);
    if (st != MB_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    float4 *hi = (float4 *)d->scratch;
    float4 *lo = (float4 *)(d->scratch + kNoallocPosBytes);
    double *partial = (double *)(d->scratch + 2 * kNoallocPosBytes);
    const double scale = 1.0 / (6.0 * kPi * eta * a);
    const int grid_pack = (int)std::min<int64_t>(ceil_div(n, 256), 1024);
    pack_hilo_kernel<false><<<grid_pack, 256, 0, s>>>(r, n, hi, lo, nullptr);
    count_launch();
    const Plan p = make_plan(n, kNT * kTPT, wall ? d->resident_wall : d->resident_free,
                             kNoallocMaxChunks);
    const int direct = p.S == 1;
    double *out = direct ? u : partial;
    const PairConsts<float> k = PairConsts<float>::make(a);
    if (wall)
        pair_f32_kernel<true, kTPT><<<p.grid, kNT, 0, s>>>(hi, lo, f, n, p.chunk, p.n_tblocks,
                                                           p.items, k, out, scale, direct);
    else
        pair_f32_kernel<false, kTPT><<<p.grid, kNT, 0, s>>>(hi, lo, f, n, p.chunk, p.n_tblocks,
                                                            p.items, k, out, scale, direct);
    count_launch();
    if (!direct) {
        const int grid = (int)std::min<int64_t>(ceil_div(3 * n, 256), 1024);
        reduce_partials_kernel<<<grid, 256, 0, s>>>(partial, n, p.S, scale, u);
        count_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_thread_err(cudaGetErrorString(e));
        return MB_ECUDA;
    }
    return MB_OK;
}
