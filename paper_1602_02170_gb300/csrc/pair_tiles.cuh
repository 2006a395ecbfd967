// Source-tile loops of the pair kernels, shared by the single-problem
// kernels (pair_matvec.cu) and the batched ones (batch.cu).
//
// One call processes one work item: the targets of target block `tb` of one
// problem against that problem's sources [j_begin, j_end).  Pointers are
// already offset to the problem; `out` receives the item's velocities at
// out + 3 i (i = target index within the problem) multiplied by `m`.
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
__device__ __forceinline__ void x2_item(float4 *__restrict__ sP, const float4 *__restrict__ hi,
                                        const float4 *__restrict__ lo,
                                        const double *__restrict__ f, int64_t n, int tb,
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
            h[hh] = hi[i];
            l[hh] = lo[i];
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
#pragma unroll 2
        for (int s = 0; s < NT; ++s) {
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
__device__ __forceinline__ void f64_item(double *__restrict__ sm, const double *__restrict__ r,
                                         const double *__restrict__ f, int64_t n, int tb,
                                         int64_t j_begin, int64_t j_end,
                                         const PairConsts<double> &k, double *__restrict__ out,
                                         double m)
{
    double *sx = sm, *sy = sm + NT, *sz = sm + 2 * NT, *sfx = sm + 3 * NT, *sfy = sm + 4 * NT,
           *sfz = sm + 5 * NT;
    const int64_t i = (int64_t)tb * NT + threadIdx.x;
    const int64_t ic = i < n ? i : n - 1;
    const double xi = r[3 * ic], yi = r[3 * ic + 1], zi = r[3 * ic + 2];
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
#pragma unroll 2
        for (int s = 0; s < NT; ++s)
            pair_accumulate<WALL, double>(xi - sx[s], yi - sy[s], zi - sz[s], zi, sz[s], sfx[s],
                                          sfy[s], sfz[s], k, ux, uy, uz);
    }
    if (i < n) {
        out[3 * i] = m * ux;
        out[3 * i + 1] = m * uy;
        out[3 * i + 2] = m * uz;
    }
}

// Double-float item: one target per thread; the same pair formula as the
// FP32 and FP64 kernels evaluated in double-float (df32.cuh).  Sources are
// staged as three float4: (x_hi, x_lo, y_hi, y_lo), (z_hi, z_lo, fx_hi,
// fx_lo), (fy_hi, fy_lo, fz_hi, fz_lo); positions come from the packed hi/lo
// arrays, forces are split from FP64 on the fly.
template <bool WALL, int NT>
__device__ __forceinline__ void df_item(float4 *__restrict__ sD, const float4 *__restrict__ hi,
                                        const float4 *__restrict__ lo,
                                        const double *__restrict__ f, int64_t n, int tb,
                                        int64_t j_begin, int64_t j_end, const PairConsts<dfl> &k,
                                        double *__restrict__ out, double m)
{
    const int64_t i = (int64_t)tb * NT + threadIdx.x;
    const int64_t ic = i < n ? i : n - 1;
    const float4 th = hi[ic], tl = lo[ic];
    const dfl xi(th.x, tl.x), yi(th.y, tl.y), zi(th.z, tl.z);
    dfl ux, uy, uz;
    for (int64_t jt = j_begin; jt < j_end; jt += NT) {
        __syncthreads();
        {
            const int64_t j = jt + threadIdx.x;
            const bool valid = j < j_end;
            const int64_t jc = valid ? j : j_begin;
            const float4 h = hi[jc], l = lo[jc];
            const dfl fx = valid ? dfl(f[3 * jc]) : dfl();
            const dfl fy = valid ? dfl(f[3 * jc + 1]) : dfl();
            const dfl fz = valid ? dfl(f[3 * jc + 2]) : dfl();
            float4 *d = sD + 3 * threadIdx.x;
            d[0] = make_float4(h.x, l.x, h.y, l.y);
            d[1] = make_float4(h.z, l.z, fx.hi, fx.lo);
            d[2] = make_float4(fy.hi, fy.lo, fz.hi, fz.lo);
        }
        __syncthreads();
#pragma unroll 1
        for (int s = 0; s < NT; ++s) {
            const float4 A = sD[3 * s], B = sD[3 * s + 1], C = sD[3 * s + 2];
            const dfl zj(B.x, B.y);
            pair_accumulate<WALL, dfl>(xi - dfl(A.x, A.y), yi - dfl(A.z, A.w), zi - zj, zi, zj,
                                       dfl(B.z, B.w), dfl(C.x, C.y), dfl(C.z, C.w), k, ux, uy, uz);
        }
    }
    if (i < n) {
        out[3 * i] = m * to_double(ux);
        out[3 * i + 1] = m * to_double(uy);
        out[3 * i + 2] = m * to_double(uz);
    }
}

}  // namespace mb
