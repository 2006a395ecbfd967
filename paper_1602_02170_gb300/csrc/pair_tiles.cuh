// Source-tile loops of the pair kernels, shared by the single-problem
// kernels (pair_matvec.cu) and the batched ones (batch.cu).
//
// One call processes one work item: the targets of target block `tb` of one
// problem against that problem's sources [j_begin, j_end).  Pointers are
// already offset to the problem; `out` receives the item's velocities at
// out + 3 i (i = target index within the problem) multiplied by `m`.  The
// non-symmetric items take the targets (n of them) from their own arrays,
// which are the source arrays themselves for a matvec and other points when
// a flow is evaluated away from the blobs.
#pragma once

#include "df32.cuh"
#include "rpy_wall.cuh"

namespace mb {

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x)
{
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// Shared-memory floats per source in the packed kernel (5 float4).
constexpr int kX2SmemFloat4PerSource = 5;

// Packed FP32 item: each thread owns 2*NP targets, held as NP float2 pairs;
// target of pair q, half h: tb*NT*2*NP + (2q + h)*NT + threadIdx.x.
// Sources are staged once per tile as duplicated float2 operands:
//   sP[5s+0] = (-x_hi, -x_hi, -y_hi, -y_hi)   sP[5s+1] = (-z_hi, -z_hi, z_hi, z_hi)
//   sP[5s+2] = (-x_lo, -x_lo, -y_lo, -y_lo)   sP[5s+3] = (-z_lo, -z_lo, f_x, f_x)
//   sP[5s+4] = (f_y, f_y, f_z, f_z)
template <bool WALL, int NP, int NT>
__device__ __forceinline__ void x2_item(float4 *__restrict__ sP, const float4 *__restrict__ thi,
                                        const float4 *__restrict__ tlo, int64_t n,
                                        const float4 *__restrict__ hi,
                                        const float4 *__restrict__ lo,
                                        const double *__restrict__ f, int tb,
                                        int64_t j_begin, int64_t j_end, const PairConsts2 &k,
                                        double *__restrict__ out, double m)
{
    float2 xh[NP], yh[NP], zh[NP], xl[NP], yl[NP], zl[NP];
    float sum[2 * NP][3], comp[2 * NP][3];
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        float4 h[2], l[2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            int64_t i = (int64_t)tb * NT * 2 * NP + (2 * q + hh) * NT + threadIdx.x;
            i = i < n ? i : n - 1;
            h[hh] = thi[i];
            l[hh] = tlo[i];
        }
        xh[q] = make_float2(h[0].x, h[1].x);
        yh[q] = make_float2(h[0].y, h[1].y);
        zh[q] = make_float2(h[0].z, h[1].z);
        xl[q] = make_float2(l[0].x, l[1].x);
        yl[q] = make_float2(l[0].y, l[1].y);
        zl[q] = make_float2(l[0].z, l[1].z);
    }
#pragma unroll
    for (int t = 0; t < 2 * NP; ++t)
#pragma unroll
        for (int c = 0; c < 3; ++c) sum[t][c] = comp[t][c] = 0.f;
    for (int64_t jt = j_begin; jt < j_end; jt += NT) {
        __syncthreads();
        {
            const int64_t j = jt + threadIdx.x;
            const bool valid = j < j_end;
            const int64_t jc = valid ? j : j_begin;
            const float4 h = hi[jc], l = lo[jc];
            const float fx = valid ? (float)f[3 * jc] : 0.f;
            const float fy = valid ? (float)f[3 * jc + 1] : 0.f;
            const float fz = valid ? (float)f[3 * jc + 2] : 0.f;
            float4 *d = sP + kX2SmemFloat4PerSource * threadIdx.x;
            d[0] = make_float4(-h.x, -h.x, -h.y, -h.y);
            d[1] = make_float4(-h.z, -h.z, h.z, h.z);
            d[2] = make_float4(-l.x, -l.x, -l.y, -l.y);
            d[3] = make_float4(-l.z, -l.z, fx, fx);
            d[4] = make_float4(fy, fy, fz, fz);
        }
        __syncthreads();
        float2 ax[NP], ay[NP], az[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) ax[q] = ay[q] = az[q] = make_float2(0.f, 0.f);
        // the staged sources of this tile (chunks may be shorter than NT)
        const int cnt = j_end - jt < NT ? (int)(j_end - jt) : NT;
#pragma unroll 2
        for (int s = 0; s < cnt; ++s) {
            const float4 *P = sP + kX2SmemFloat4PerSource * s;
            const float4 P0 = P[0], P1 = P[1], P2 = P[2], P3 = P[3], P4 = P[4];
            const float2 nxh = make_float2(P0.x, P0.y), nyh = make_float2(P0.z, P0.w);
            const float2 nzh = make_float2(P1.x, P1.y), zj = make_float2(P1.z, P1.w);
            const float2 nxl = make_float2(P2.x, P2.y), nyl = make_float2(P2.z, P2.w);
            const float2 nzl = make_float2(P3.x, P3.y), fx = make_float2(P3.z, P3.w);
            const float2 fy = make_float2(P4.x, P4.y), fz = make_float2(P4.z, P4.w);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float2 dx = add2(add2(xh[q], nxh), add2(xl[q], nxl));
                const float2 dy = add2(add2(yh[q], nyh), add2(yl[q], nyl));
                const float2 dz = add2(add2(zh[q], nzh), add2(zl[q], nzl));
                const float2 dxy2 = fma2(dy, dy, fma2(dx, dx, k.tiny));
                pair_accumulate2<WALL>(dx, dy, dz, dxy2, zh[q], zj, fx, fy, fz, k, ax[q], ay[q],
                                       az[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            kahan_add(sum[2 * q][0], comp[2 * q][0], ax[q].x);
            kahan_add(sum[2 * q][1], comp[2 * q][1], ay[q].x);
            kahan_add(sum[2 * q][2], comp[2 * q][2], az[q].x);
            kahan_add(sum[2 * q + 1][0], comp[2 * q + 1][0], ax[q].y);
            kahan_add(sum[2 * q + 1][1], comp[2 * q + 1][1], ay[q].y);
            kahan_add(sum[2 * q + 1][2], comp[2 * q + 1][2], az[q].y);
        }
    }
#pragma unroll
    for (int t = 0; t < 2 * NP; ++t) {
        const int64_t i = (int64_t)tb * NT * 2 * NP + t * NT + threadIdx.x;
        if (i < n) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                out[3 * i + c] = m * ((double)sum[t][c] - (double)comp[t][c]);
        }
    }
}

// FP64 item: one target per thread, sources staged as six double arrays.
template <bool WALL, int NT>
__device__ __forceinline__ void f64_item(double *__restrict__ sm, const double *__restrict__ tr,
                                         int64_t n, const double *__restrict__ r,
                                         const double *__restrict__ f, int tb,
                                         int64_t j_begin, int64_t j_end,
                                         const PairConsts<double> &k, double *__restrict__ out,
                                         double m)
{
    double *sx = sm, *sy = sm + NT, *sz = sm + 2 * NT, *sfx = sm + 3 * NT, *sfy = sm + 4 * NT,
           *sfz = sm + 5 * NT;
    const int64_t i = (int64_t)tb * NT + threadIdx.x;
    const int64_t ic = i < n ? i : n - 1;
    const double xi = tr[3 * ic], yi = tr[3 * ic + 1], zi = tr[3 * ic + 2];
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int64_t jt = j_begin; jt < j_end; jt += NT) {
        __syncthreads();
        {
            const int64_t j = jt + threadIdx.x;
            const bool valid = j < j_end;
            const int64_t jc = valid ? j : j_begin;
            sx[threadIdx.x] = r[3 * jc];
            sy[threadIdx.x] = r[3 * jc + 1];
            sz[threadIdx.x] = r[3 * jc + 2];
            sfx[threadIdx.x] = valid ? f[3 * jc] : 0.0;
            sfy[threadIdx.x] = valid ? f[3 * jc + 1] : 0.0;
            sfz[threadIdx.x] = valid ? f[3 * jc + 2] : 0.0;
        }
        __syncthreads();
        // the staged sources of this tile (chunks may be shorter than NT)
        const int cnt = j_end - jt < NT ? (int)(j_end - jt) : NT;
#pragma unroll 2
        for (int s = 0; s < cnt; ++s)
            pair_accumulate<WALL, double>(xi - sx[s], yi - sy[s], zi - sz[s], zi, sz[s], sfx[s],
                                          sfy[s], sfz[s], k, ux, uy, uz);
    }
    if (i < n) {
        out[3 * i] = m * ux;
        out[3 * i + 1] = m * uy;
        out[3 * i + 2] = m * uz;
    }
}

// Symmetric packed item over block pair (I, J), I <= J, blocks of 2*NT blobs
// (two targets per thread, as in x2_item with NP = 1).  Each unordered pair
// is evaluated once.  Forward contributions accumulate in the thread's
// registers (tile sums folded Kahan-style).  Reverse contributions use a
// rotating schedule inside each group of 32 staged sources: at step t lane l
// pairs its targets with source (l + t) mod 32, adds the reverse term into a
// packed accumulator, and passes that accumulator to lane l - 1; after 32
// steps lane l holds source l's sum over the warp's 64 targets (no per-source
// reduction).  The warps' sums are added in a fixed order in shared memory
// and then to u with FP64 atomics.  Diagonal items (I == J) run forward only
// over all ordered pairs.  u must be zeroed beforehand and receives
// scale * M f.
//
// FAR (off-diagonal block pairs whose bounding boxes are farther apart than
// both 2a and 2^18 ulp of the largest coordinate): the separations take the
// hi parts alone, whose rounding then moves a separation by at most 2^-18 of
// itself, and the overlap test is left out.
template <bool WALL, int NT, bool FAR = false>
__device__ __forceinline__ void x2sym_item(float4 *__restrict__ sP, float *__restrict__ sRev,
                                           const float4 *__restrict__ hi,
                                           const float4 *__restrict__ lo,
                                           const double *__restrict__ f, int64_t n, int64_t I,
                                           int64_t J, const PairConsts2 &k,
                                           double *__restrict__ u, double scale)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool diag = I == J;
    const int64_t ia = I * 2 * NT + threadIdx.x, ib = ia + NT;
    float2 xh, yh, zh, xl, yl, zl, fix, fiy, fiz;
    {
        const int64_t ca = ia < n ? ia : n - 1, cb = ib < n ? ib : n - 1;
        const float4 ha = hi[ca], hb = hi[cb], la = lo[ca], lb = lo[cb];
        xh = make_float2(ha.x, hb.x); yh = make_float2(ha.y, hb.y); zh = make_float2(ha.z, hb.z);
        xl = make_float2(la.x, lb.x); yl = make_float2(la.y, lb.y); zl = make_float2(la.z, lb.z);
        // padding targets carry no force, so their reverse contributions vanish
        fix = make_float2(ia < n ? (float)f[3 * ia] : 0.f, ib < n ? (float)f[3 * ib] : 0.f);
        fiy = make_float2(ia < n ? (float)f[3 * ia + 1] : 0.f, ib < n ? (float)f[3 * ib + 1] : 0.f);
        fiz = make_float2(ia < n ? (float)f[3 * ia + 2] : 0.f, ib < n ? (float)f[3 * ib + 2] : 0.f);
    }
    float sum[2][3], comp[2][3];
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int c = 0; c < 3; ++c) sum[t][c] = comp[t][c] = 0.f;
    for (int sub = 0; sub < 2; ++sub) {
        const int64_t j0 = J * 2 * NT + sub * NT;
        if (j0 >= n) break;
        __syncthreads();
        {
            const int64_t j = j0 + threadIdx.x;
            const bool valid = j < n;
            const int64_t jc = valid ? j : j0;
            const float4 h = hi[jc], l = lo[jc];
            const float fx = valid ? (float)f[3 * jc] : 0.f;
            const float fy = valid ? (float)f[3 * jc + 1] : 0.f;
            const float fz = valid ? (float)f[3 * jc + 2] : 0.f;
            float4 *d = sP + kX2SmemFloat4PerSource * threadIdx.x;
            d[0] = make_float4(-h.x, -h.x, -h.y, -h.y);
            d[1] = make_float4(-h.z, -h.z, h.z, h.z);
            d[2] = make_float4(-l.x, -l.x, -l.y, -l.y);
            d[3] = make_float4(-l.z, -l.z, fx, fx);
            d[4] = make_float4(fy, fy, fz, fz);
        }
        __syncthreads();
        float2 ax = make_float2(0.f, 0.f), ay = ax, az = ax;
        if (diag) {
#pragma unroll 2
            for (int s = 0; s < NT; ++s) {
                const float4 *P = sP + kX2SmemFloat4PerSource * s;
                const float4 P0 = P[0], P1 = P[1], P2 = P[2], P3 = P[3], P4 = P[4];
                const float2 dx = add2(add2(xh, make_float2(P0.x, P0.y)), add2(xl, make_float2(P2.x, P2.y)));
                const float2 dy = add2(add2(yh, make_float2(P0.z, P0.w)), add2(yl, make_float2(P2.z, P2.w)));
                const float2 dz = add2(add2(zh, make_float2(P1.x, P1.y)), add2(zl, make_float2(P3.x, P3.y)));
                const float2 dxy2 = fma2(dy, dy, fma2(dx, dx, k.tiny));
                pair_accumulate2<WALL>(dx, dy, dz, dxy2, zh, make_float2(P1.z, P1.w),
                                       make_float2(P3.z, P3.w), make_float2(P4.x, P4.y),
                                       make_float2(P4.z, P4.w), k, ax, ay, az);
            }
        } else {
            for (int g = 0; g < NT / 32; ++g) {
                float2 rx = make_float2(0.f, 0.f), ry = rx, rz = rx;
#pragma unroll 2
                for (int t = 0; t < 32; ++t) {
                    const int s = g * 32 + ((lane + t) & 31);
                    const float4 *P = sP + kX2SmemFloat4PerSource * s;
                    const float4 P0 = P[0], P1 = P[1], P3 = P[3], P4 = P[4];
                    float2 dx, dy, dz;
                    if (FAR) {
                        dx = add2(xh, make_float2(P0.x, P0.y));
                        dy = add2(yh, make_float2(P0.z, P0.w));
                        dz = add2(zh, make_float2(P1.x, P1.y));
                    } else {
                        const float4 P2 = P[2];
                        dx = add2(add2(xh, make_float2(P0.x, P0.y)), add2(xl, make_float2(P2.x, P2.y)));
                        dy = add2(add2(yh, make_float2(P0.z, P0.w)), add2(yl, make_float2(P2.z, P2.w)));
                        dz = add2(add2(zh, make_float2(P1.x, P1.y)), add2(zl, make_float2(P3.x, P3.y)));
                    }
                    const float2 dxy2 = fma2(dy, dy, fma2(dx, dx, k.tiny));
                    pair_sym2<WALL, FAR>(dx, dy, dz, dxy2, zh, make_float2(P1.z, P1.w),
                                         make_float2(P3.z, P3.w), make_float2(P4.x, P4.y),
                                         make_float2(P4.z, P4.w), fix, fiy, fiz, k, ax, ay, az, rx,
                                         ry, rz);
                    // hand the accumulator to lane - 1, which meets this source next step
                    const int from = (lane + 1) & 31;
                    rx.x = __shfl_sync(0xffffffffu, rx.x, from);
                    rx.y = __shfl_sync(0xffffffffu, rx.y, from);
                    ry.x = __shfl_sync(0xffffffffu, ry.x, from);
                    ry.y = __shfl_sync(0xffffffffu, ry.y, from);
                    rz.x = __shfl_sync(0xffffffffu, rz.x, from);
                    rz.y = __shfl_sync(0xffffffffu, rz.y, from);
                }
                float *o3 = sRev + 3 * (warp * NT + g * 32 + lane);
                o3[0] = rx.x + rx.y;
                o3[1] = ry.x + ry.y;
                o3[2] = rz.x + rz.y;
            }
        }
        kahan_add(sum[0][0], comp[0][0], ax.x);
        kahan_add(sum[0][1], comp[0][1], ay.x);
        kahan_add(sum[0][2], comp[0][2], az.x);
        kahan_add(sum[1][0], comp[1][0], ax.y);
        kahan_add(sum[1][1], comp[1][1], ay.y);
        kahan_add(sum[1][2], comp[1][2], az.y);
        if (!diag) {
            __syncthreads();
            const int64_t j = j0 + threadIdx.x;
            if (j < n) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float acc = 0.f;
#pragma unroll
                    for (int w = 0; w < NW; ++w) acc += sRev[3 * (w * NT + threadIdx.x) + c];
                    atomicAdd(u + 3 * j + c, scale * (double)acc);
                }
            }
        }
    }
    if (ia < n)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            atomicAdd(u + 3 * ia + c, scale * ((double)sum[0][c] - (double)comp[0][c]));
    if (ib < n)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            atomicAdd(u + 3 * ib + c, scale * ((double)sum[1][c] - (double)comp[1][c]));
}

// FP64 forms of the FP32-operand operations of df32.cuh, so that the
// regrouped pair formula below serves FP64 and double-float alike.
__device__ __forceinline__ double mulf(double a, float c) { return a * (double)c; }
__device__ __forceinline__ double mul_pow2(double a, float c) { return a * (double)c; }
__device__ __forceinline__ double addf(double a, float c) { return a + (double)c; }

// pair_sym (both directions of one unordered pair) for FP64 and
// double-float operands, with the wall polynomials regrouped so that
// constants exact in FP32 (2, 4, 6, 10, 12, 20, ...) take the cheaper
// FP32-operand products of df32.cuh and the factors of 1/3 are applied to
// three shared monomials once:
//   T1 = E t2,  t4_3 = t4 / 3,  t2_3 = t2 / 3,  T2_3 = E t4 / 3,
//   f1 = 2 (T1 - p + t4_3 - t2_3) - 10 T2_3 - 1
//   f2 = F2 - 1,  F2 = 2 (3 p - 5 T1 + t2) + 10 (7 T2_3 - t4_3)
//   f3 = 2 hs + e3 (20 t4_3 - 2 F2)
//   f4 = 2 hs - 20 e3 t4_3
//   f5 = 4 (15 T2_3 - 2 t4_3 - hs^2 - T1)
// (the f1..f5 of rpy_wall.cuh term by term; the bracket of f3,
// t2 (20E - 4) + t4 (40/3 - 140E/3) - 12p, equals 20 t4 / 3 - 2 (f2 + 1)),
// and f2 / rho^2, f3 / rho, f4 / rho formed once for both directions as in
// pair_sym2.
//
// FAR (double-float, block pairs whose boxes are at least 64 a apart, so
// that t4 = (a / rho)^4 < 2^-24 and no pair overlaps): the terms carrying t4
// are summed in FP32 and added to the double-float rest once per
// polynomial; their rounding is then below 2^-24 t4 of the polynomial,
// under the double-float rounding of the other terms.
template <bool WALL, typename T, bool FAR = false>
__device__ __forceinline__ void pair_sym_rg(T dx, T dy, T dz, T zi, T zj, T fx, T fy, T fz, T gx,
                                            T gy, T gz, const PairConsts<T> &k, T &ux, T &uy,
                                            T &uz, T &vx, T &vy, T &vz)
{
    const T dxy2 = dx * dx + dy * dy;
    const T r2 = mb_max(dz * dz + dxy2, k.tiny);
    const T inv = mb_rsqrt(r2);
    const T inv2 = inv * inv;
    T C = inv * (k.c1 + k.c2 * inv2);
    T D = inv * inv2 * (k.c3 + k.c4 * inv2);
    if (!FAR && r2 < k.four_a2) {
        C = T(1) - k.k1 * (r2 * inv);
        D = k.k2 * inv;
    }
    const T rf_xy = dx * fx + dy * fy;
    const T g = D * (rf_xy + dz * fz);
    const T rb_xy = dx * gx + dy * gy;
    const T gb = D * (rb_xy + dz * gz);
    if (!WALL) {
        acc_add(ux, C * fx + g * dx);
        acc_add(uy, C * fy + g * dy);
        acc_add(uz, C * fz + g * dz);
        acc_add(vx, C * gx + gb * dx);
        acc_add(vy, C * gy + gb * dy);
        acc_add(vz, C * gz + gb * dz);
        return;
    }
    constexpr T third(1.0 / 3.0);
    const T R3 = zi + zj;
    const T invR = mb_rsqrt(R3 * R3 + dxy2);
    const T invR2 = invR * invR;
    const T hs = zj * invR;
    const T ht = zi * invR;
    const T e3 = hs + ht;
    const T E = e3 * e3;
    const T t2 = k.a2 * invR2;
    const T p = hs * ht;
    const T T1 = E * t2;
    const T t2_3 = t2 * third;
    const T hs2 = mul_pow2(hs, 2.f);
    T f1, F2, f3, f4, f5;
    if constexpr (FAR) {
        // the t4 terms in FP32 (t4 / 3, E t4 / 3 from the high parts)
        const float t4_3f = hi_part(t2) * hi_part(t2) * (1.f / 3.f);
        const float T2_3f = hi_part(E) * t4_3f, e3t4_3f = hi_part(e3) * t4_3f;
        f1 = addf(addf(mul_pow2(T1 + (-p) + (-t2_3), 2.f), -1.f), 2.f * t4_3f - 10.f * T2_3f);
        F2 = addf(mul_pow2(mulf(p, 3.f) + mulf(T1, -5.f) + t2, 2.f), 10.f * (7.f * T2_3f - t4_3f));
        f3 = addf(hs2 + e3 * mul_pow2(F2, -2.f), 20.f * e3t4_3f);
        f4 = addf(hs2, -20.f * e3t4_3f);
        f5 = addf(mul_pow2((-(hs * hs)) + (-T1), 4.f), 4.f * (15.f * T2_3f - 2.f * t4_3f));
    } else {
        const T t4 = t2 * t2;
        const T t4_3 = t4 * third;
        const T T2_3 = E * t4_3;
        f1 = addf(mul_pow2(T1 + (-p) + t4_3 + (-t2_3), 2.f) + mulf(T2_3, -10.f), -1.f);
        F2 = mul_pow2(mulf(p, 3.f) + mulf(T1, -5.f) + t2, 2.f) +
             mulf(mulf(T2_3, 7.f) + (-t4_3), 10.f);
        f3 = hs2 + e3 * (mulf(t4_3, 20.f) + mul_pow2(F2, -2.f));
        f4 = hs2 + mulf(e3 * t4_3, -20.f);
        f5 = mul_pow2(mulf(T2_3, 15.f) + mul_pow2(t4_3, -2.f) + (-(hs * hs)) + (-T1), 4.f);
    }
    const T f2 = addf(F2, -1.f);
    const T s = k.sw * invR;
    const T Cx = C + s * f1;
    const T A2 = f2 * invR2;
    const T A3 = f3 * invR;
    const T A4 = f4 * invR;
    // forward: M_ij f_j
    const T RF = rf_xy + R3 * fz;
    const T gw = A2 * RF + A3 * fz;
    const T kz = A4 * RF + f5 * fz;
    const T Gx = g + s * gw;
    acc_add(ux, Cx * fx + Gx * dx);
    acc_add(uy, Cx * fy + Gx * dy);
    acc_add(uz, Cx * fz + g * dz + s * (gw * R3 + kz));
    // reverse: M_ij^T f_i (f3 and f4 exchange roles)
    const T RB = rb_xy + R3 * gz;
    const T gwb = A2 * RB + A4 * gz;
    const T kzb = A3 * RB + f5 * gz;
    const T Gb = gb + s * gwb;
    acc_add(vx, Cx * gx + Gb * dx);
    acc_add(vy, Cx * gy + Gb * dy);
    acc_add(vz, Cx * gz + gb * dz + s * (gwb * R3 + kzb));
}

// Symmetric double-float item over block pair (I, J), I <= J, blocks of NT
// blobs, one target per thread; the rotating reverse accumulators of
// x2sym_item in double-float.  Sources are staged as three float4 (x_hi,
// x_lo, y_hi, y_lo), (z_hi, z_lo, fx_hi, fx_lo), (fy_hi, fy_lo, fz_hi,
// fz_lo): a 48-byte stride, so the rotated reads stay conflict-free.
// sRev holds NT * 3 doubles: each warp adds its per-source sums with shared-
// memory atomics.  u must be zeroed and receives scale * M f.
template <bool WALL, int NT, bool FAR = false>
__device__ __forceinline__ void dfsym_item(float4 *__restrict__ sD, double *__restrict__ sRev,
                                           const float4 *__restrict__ hi,
                                           const float4 *__restrict__ lo,
                                           const double *__restrict__ f, int64_t n, int64_t I,
                                           int64_t J, const PairConsts<dfl> &k,
                                           double *__restrict__ u, double scale)
{
    const int lane = threadIdx.x & 31;
    const bool diag = I == J;
    const int64_t i = I * NT + threadIdx.x;
    const int64_t ic = i < n ? i : n - 1;
    const float4 th = hi[ic], tl = lo[ic];
    const dfl xi(th.x, tl.x), yi(th.y, tl.y), zi(th.z, tl.z);
    const dfl gx = i < n ? dfl(f[3 * i]) : dfl(), gy = i < n ? dfl(f[3 * i + 1]) : dfl(),
              gz = i < n ? dfl(f[3 * i + 2]) : dfl();
    dfl ux, uy, uz;
    const int64_t j0 = J * NT;
    __syncthreads();
    {
        const int64_t j = j0 + threadIdx.x;
        const bool valid = j < n;
        const int64_t jc = valid ? j : j0;
        const float4 h = hi[jc], l = lo[jc];
        const dfl fx = valid ? dfl(f[3 * jc]) : dfl();
        const dfl fy = valid ? dfl(f[3 * jc + 1]) : dfl();
        const dfl fz = valid ? dfl(f[3 * jc + 2]) : dfl();
        float4 *d = sD + 3 * threadIdx.x;
        d[0] = make_float4(h.x, l.x, h.y, l.y);
        d[1] = make_float4(h.z, l.z, fx.hi, fx.lo);
        d[2] = make_float4(fy.hi, fy.lo, fz.hi, fz.lo);
        sRev[3 * threadIdx.x] = sRev[3 * threadIdx.x + 1] = sRev[3 * threadIdx.x + 2] = 0.0;
    }
    __syncthreads();
    if (diag) {
#pragma unroll 1
        for (int s = 0; s < NT; ++s) {
            const float4 A = sD[3 * s], B = sD[3 * s + 1], C = sD[3 * s + 2];
            const dfl zj(B.x, B.y);
            pair_accumulate<WALL, dfl>(xi - dfl(A.x, A.y), yi - dfl(A.z, A.w), zi - zj, zi, zj,
                                       dfl(B.z, B.w), dfl(C.x, C.y), dfl(C.z, C.w), k, ux, uy, uz);
        }
    } else {
        for (int g = 0; g < NT / 32; ++g) {
            dfl vx, vy, vz;
#pragma unroll 1
            for (int t = 0; t < 32; ++t) {
                const int s = g * 32 + ((lane + t) & 31);
                const float4 A = sD[3 * s], B = sD[3 * s + 1], C = sD[3 * s + 2];
                const dfl zj(B.x, B.y);
                pair_sym_rg<WALL, dfl, FAR>(xi - dfl(A.x, A.y), yi - dfl(A.z, A.w), zi - zj, zi, zj,
                                  dfl(B.z, B.w), dfl(C.x, C.y), dfl(C.z, C.w), gx, gy, gz, k, ux,
                                  uy, uz, vx, vy, vz);
                const int from = (lane + 1) & 31;
                vx.hi = __shfl_sync(0xffffffffu, vx.hi, from);
                vx.lo = __shfl_sync(0xffffffffu, vx.lo, from);
                vy.hi = __shfl_sync(0xffffffffu, vy.hi, from);
                vy.lo = __shfl_sync(0xffffffffu, vy.lo, from);
                vz.hi = __shfl_sync(0xffffffffu, vz.hi, from);
                vz.lo = __shfl_sync(0xffffffffu, vz.lo, from);
            }
            double *o3 = sRev + 3 * (g * 32 + lane);
            atomicAdd(o3, to_double(vx));
            atomicAdd(o3 + 1, to_double(vy));
            atomicAdd(o3 + 2, to_double(vz));
            // the forward sums take sloppy additions: renormalised every 32 terms
            renorm(ux);
            renorm(uy);
            renorm(uz);
        }
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        if (j < n) {
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(u + 3 * j + c, scale * sRev[3 * threadIdx.x + c]);
        }
    }
    if (i < n) {
        atomicAdd(u + 3 * i, scale * to_double(ux));
        atomicAdd(u + 3 * i + 1, scale * to_double(uy));
        atomicAdd(u + 3 * i + 2, scale * to_double(uz));
    }
}

// FP64 symmetric item over block pair (I, J), I <= J, blocks of NT blobs,
// one target per thread: the scheme of dfsym_item in FP64.  Sources are
// staged as six FP64 arrays (lanes read consecutive sources: no bank
// conflicts); each unordered pair is evaluated once for both blobs, the
// reverse sums rotate through the warp (lane l holds source l's sum after 32
// steps) and reach u with FP64 atomics, so u must be zeroed beforehand.
// Diagonal items run forward only over all ordered pairs.
template <bool WALL, int NT>
__device__ __forceinline__ void f64sym_item(double *__restrict__ sm, const double *__restrict__ r,
                                            const double *__restrict__ f, int64_t n, int64_t I,
                                            int64_t J, const PairConsts<double> &k,
                                            double *__restrict__ u, double scale)
{
    double *sx = sm, *sy = sm + NT, *sz = sm + 2 * NT, *sfx = sm + 3 * NT, *sfy = sm + 4 * NT,
           *sfz = sm + 5 * NT, *sRev = sm + 6 * NT;
    const int lane = threadIdx.x & 31;
    const bool diag = I == J;
    const int64_t i = I * NT + threadIdx.x;
    const int64_t ic = i < n ? i : n - 1;
    const double xi = r[3 * ic], yi = r[3 * ic + 1], zi = r[3 * ic + 2];
    const double gx = i < n ? f[3 * i] : 0.0, gy = i < n ? f[3 * i + 1] : 0.0,
                 gz = i < n ? f[3 * i + 2] : 0.0;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    const int64_t j0 = J * NT;
    __syncthreads();
    {
        const int64_t j = j0 + threadIdx.x;
        const bool valid = j < n;
        const int64_t jc = valid ? j : j0;
        sx[threadIdx.x] = r[3 * jc];
        sy[threadIdx.x] = r[3 * jc + 1];
        sz[threadIdx.x] = r[3 * jc + 2];
        sfx[threadIdx.x] = valid ? f[3 * jc] : 0.0;
        sfy[threadIdx.x] = valid ? f[3 * jc + 1] : 0.0;
        sfz[threadIdx.x] = valid ? f[3 * jc + 2] : 0.0;
        sRev[3 * threadIdx.x] = sRev[3 * threadIdx.x + 1] = sRev[3 * threadIdx.x + 2] = 0.0;
    }
    __syncthreads();
    if (diag) {
#pragma unroll 1
        for (int s = 0; s < NT; ++s)
            pair_accumulate<WALL, double>(xi - sx[s], yi - sy[s], zi - sz[s], zi, sz[s], sfx[s],
                                          sfy[s], sfz[s], k, ux, uy, uz);
    } else {
        for (int g = 0; g < NT / 32; ++g) {
            double vx = 0.0, vy = 0.0, vz = 0.0;
#pragma unroll 1
            for (int t = 0; t < 32; ++t) {
                const int s = g * 32 + ((lane + t) & 31);
                pair_sym_rg<WALL, double>(xi - sx[s], yi - sy[s], zi - sz[s], zi, sz[s], sfx[s],
                                          sfy[s], sfz[s], gx, gy, gz, k, ux, uy, uz, vx, vy, vz);
                const int from = (lane + 1) & 31;
                vx = __shfl_sync(0xffffffffu, vx, from);
                vy = __shfl_sync(0xffffffffu, vy, from);
                vz = __shfl_sync(0xffffffffu, vz, from);
            }
            double *o3 = sRev + 3 * (g * 32 + lane);
            atomicAdd(o3, vx);
            atomicAdd(o3 + 1, vy);
            atomicAdd(o3 + 2, vz);
        }
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        if (j < n) {
#pragma unroll
            for (int c = 0; c < 3; ++c) atomicAdd(u + 3 * j + c, scale * sRev[3 * threadIdx.x + c]);
        }
    }
    if (i < n) {
        atomicAdd(u + 3 * i, scale * ux);
        atomicAdd(u + 3 * i + 1, scale * uy);
        atomicAdd(u + 3 * i + 2, scale * uz);
    }
}

}  // namespace mb

