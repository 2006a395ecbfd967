// Device-side blob-blob mobility of the wall-corrected RPY tensor.
//
// Everything here is in units of (6 pi eta a)^-1; callers scale at the end.
//
// Free space (Eq. RPYTensor), with d = r_i - r_j, r = |d|:
//   r >  2a: C I + D' d d^T,  C = (3a/4)/r + (a^3/2)/r^3,
//                             D' = (3a/4)/r^3 - (3a^3/2)/r^5
//   r <= 2a: C = 1 - 9r/(32a), D' = (3/(32a))/r
// (D' is C2/r^2 or C4/r^2, so that D' (d.f) d = C2 (dhat.f) dhat.)
//
// Single no-slip wall at z = 0 (Section 2.1.1): the image part of Blake's
// Green's function with the Faxen operator (1 + a^2/6 Lap) applied at both
// blobs.  Writing R = r_i - (x_j, y_j, -z_j), rho = |R|, e = R/rho,
// hs = z_j/rho, ht = z_i/rho, e3 = hs + ht, E = e3^2, p = hs*ht,
// t2 = a^2/rho^2, t4 = t2^2, that correction is, for unit viscosity,
//   8 pi rho W_ab = f1 d_ab + f2 e_a e_b + f3 e_a d_b3 + f4 d_a3 e_b + f5 d_a3 d_b3
// with (a = velocity component, b = force component)
//   f1 = -1 - 2p + t2 (2E - 2/3)  + t4 (2/3 - 10E/3)
//   f2 = -1 + 6p + t2 (2 - 10E)   + t4 (70E/3 - 10/3)
//   f3 = 2hs + e3 [t2 (20E - 4) + t4 (40/3 - 140E/3) - 12p]
//   f4 = 2hs - (20/3) e3 t4
//   f5 = -4hs^2 - 4E t2 + t4 (20E - 8/3)
// (derived by hand from the two Faxen operators acting on Blake's image
// system; the self term i = j reduces to the Rotne-Prager-Blake self
// mobilities).  In units of (6 pi eta a)^-1 the prefactor 1/(8 pi rho)
// becomes (3a/4)/rho.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace mb {

// Per-call constants of the pair interaction (units of (6 pi eta a)^-1).
template <typename T>
struct PairConsts {
    T a2;       // a^2
    T four_a2;  // 4 a^2: r^2 below this takes the overlap branch
    T c1, c2;   // far C  = inv (c1 + c2 inv^2)
    T c3, c4;   // far D' = inv^3 (c3 + c4 inv^2)
    T k1, k2;   // near C = 1 - k1 r, D' = k2 inv
    T sw;       // wall prefactor 3a/4
    T tiny;     // floor on r^2 (coincident blobs, including i = j)

    __host__ static PairConsts make(double a)
    {
        PairConsts k;
        k.a2 = T(a * a);
        k.four_a2 = T(4.0 * a * a);
        k.c1 = T(0.75 * a);
        k.c2 = T(0.5 * a * a * a);
        k.c3 = T(0.75 * a);
        k.c4 = T(-1.5 * a * a * a);
        k.k1 = T(9.0 / (32.0 * a));
        k.k2 = T(3.0 / (32.0 * a));
        k.sw = T(0.75 * a);
        k.tiny = std::is_same<T, double>::value ? T(1e-300) : T(1e-30);
        return k;
    }
};

__device__ __forceinline__ float mb_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double mb_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float mb_max(float x, float y) { return fmaxf(x, y); }
__device__ __forceinline__ double mb_max(double x, double y) { return fmax(x, y); }

// Accumulate u += M_ij f_j for one pair, given the separation d = r_i - r_j
// (already formed by the caller, possibly from hi/lo parts), the heights
// zi, zj and the source force f.  WALL selects the wall correction.
template <bool WALL, typename T>
__device__ __forceinline__ void pair_accumulate(T dx, T dy, T dz, T zi, T zj, T fx, T fy, T fz,
                                                const PairConsts<T> &k, T &ux, T &uy, T &uz)
{
    const T dxy2 = dx * dx + dy * dy;
    const T r2 = mb_max(dz * dz + dxy2, k.tiny);
    const T inv = mb_rsqrt(r2);
    const T inv2 = inv * inv;
    T C = inv * (k.c1 + k.c2 * inv2);
    T D = inv * inv2 * (k.c3 + k.c4 * inv2);
    if (r2 < k.four_a2) {  // overlapping blobs (rare): regularised branch
        C = T(1) - k.k1 * (r2 * inv);
        D = k.k2 * inv;
    }
    const T rf_xy = dx * fx + dy * fy;
    const T g = D * (rf_xy + dz * fz);
    if (!WALL) {
        ux += C * fx + g * dx;
        uy += C * fy + g * dy;
        uz += C * fz + g * dz;
        return;
    }
    const T R3 = zi + zj;
    const T invR = mb_rsqrt(R3 * R3 + dxy2);
    const T hs = zj * invR;
    const T ht = zi * invR;
    const T e3 = hs + ht;
    const T E = e3 * e3;
    const T t2 = k.a2 * (invR * invR);
    const T t4 = t2 * t2;
    const T p = hs * ht;
    const T f1 = T(-1) - T(2) * p + t2 * (T(2) * E - T(2.0 / 3.0)) + t4 * (T(2.0 / 3.0) - T(10.0 / 3.0) * E);
    const T f2 = T(-1) + T(6) * p + t2 * (T(2) - T(10) * E) + t4 * (T(70.0 / 3.0) * E - T(10.0 / 3.0));
    const T f3 = T(2) * hs + e3 * (t2 * (T(20) * E - T(4)) + t4 * (T(40.0 / 3.0) - T(140.0 / 3.0) * E) - T(12) * p);
    const T f4 = T(2) * hs - T(20.0 / 3.0) * e3 * t4;
    const T f5 = T(-4) * hs * hs - T(4) * E * t2 + t4 * (T(20) * E - T(8.0 / 3.0));
    const T eF = (rf_xy + R3 * fz) * invR;
    const T gw = (f2 * eF + f3 * fz) * invR;
    const T kz = f4 * eF + f5 * fz;
    const T s = k.sw * invR;
    const T Cx = C + s * f1;
    const T Gx = g + s * gw;
    ux += Cx * fx + Gx * dx;
    uy += Cx * fy + Gx * dy;
    uz += Cx * fz + g * dz + s * (gw * R3 + kz);
}

// Both directions of one unordered pair (scalar types: FP64, double-float):
// u_i += M_ij f_j and v_j += M_ij^T f_i (f3 and f4 exchange roles in the
// transpose).
template <bool WALL, typename T>
__device__ __forceinline__ void pair_sym(T dx, T dy, T dz, T zi, T zj, T fx, T fy, T fz, T gx,
                                         T gy, T gz, const PairConsts<T> &k, T &ux, T &uy, T &uz,
                                         T &vx, T &vy, T &vz)
{
    const T dxy2 = dx * dx + dy * dy;
    const T r2 = mb_max(dz * dz + dxy2, k.tiny);
    const T inv = mb_rsqrt(r2);
    const T inv2 = inv * inv;
    T C = inv * (k.c1 + k.c2 * inv2);
    T D = inv * inv2 * (k.c3 + k.c4 * inv2);
    if (r2 < k.four_a2) {
        C = T(1) - k.k1 * (r2 * inv);
        D = k.k2 * inv;
    }
    const T rf_xy = dx * fx + dy * fy;
    const T g = D * (rf_xy + dz * fz);
    const T rb_xy = dx * gx + dy * gy;
    const T gb = D * (rb_xy + dz * gz);
    if (!WALL) {
        ux += C * fx + g * dx;
        uy += C * fy + g * dy;
        uz += C * fz + g * dz;
        vx += C * gx + gb * dx;
        vy += C * gy + gb * dy;
        vz += C * gz + gb * dz;
        return;
    }
    const T R3 = zi + zj;
    const T invR = mb_rsqrt(R3 * R3 + dxy2);
    const T hs = zj * invR;
    const T ht = zi * invR;
    const T e3 = hs + ht;
    const T E = e3 * e3;
    const T t2 = k.a2 * (invR * invR);
    const T t4 = t2 * t2;
    const T p = hs * ht;
    const T f1 = T(-1) - T(2) * p + t2 * (T(2) * E - T(2.0 / 3.0)) + t4 * (T(2.0 / 3.0) - T(10.0 / 3.0) * E);
    const T f2 = T(-1) + T(6) * p + t2 * (T(2) - T(10) * E) + t4 * (T(70.0 / 3.0) * E - T(10.0 / 3.0));
    const T f3 = T(2) * hs + e3 * (t2 * (T(20) * E - T(4)) + t4 * (T(40.0 / 3.0) - T(140.0 / 3.0) * E) - T(12) * p);
    const T f4 = T(2) * hs - T(20.0 / 3.0) * e3 * t4;
    const T f5 = T(-4) * hs * hs - T(4) * E * t2 + t4 * (T(20) * E - T(8.0 / 3.0));
    const T s = k.sw * invR;
    const T Cx = C + s * f1;
    const T eF = (rf_xy + R3 * fz) * invR;
    const T gw = (f2 * eF + f3 * fz) * invR;
    const T kz = f4 * eF + f5 * fz;
    const T Gx = g + s * gw;
    ux += Cx * fx + Gx * dx;
    uy += Cx * fy + Gx * dy;
    uz += Cx * fz + g * dz + s * (gw * R3 + kz);
    const T eB = (rb_xy + R3 * gz) * invR;
    const T gwb = (f2 * eB + f4 * gz) * invR;
    const T kzb = f3 * eB + f5 * gz;
    const T Gb = gb + s * gwb;
    vx += Cx * gx + Gb * dx;
    vy += Cx * gy + Gb * dy;
    vz += Cx * gz + gb * dz + s * (gwb * R3 + kzb);
}

// Full 3x3 block M_ij in FP64, units of (6 pi eta a)^-1, row-major
// m[3*alpha + beta] (alpha = velocity component of i, beta = force
// component of j).  Used to assemble the per-body blocks of the
// preconditioner.
template <bool WALL>
__device__ __forceinline__ void block_f64(const double *ri, const double *rj,
                                          const PairConsts<double> &k, double m[9])
{
    const double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        double u[3] = {0.0, 0.0, 0.0};
        const double f[3] = {b == 0 ? 1.0 : 0.0, b == 1 ? 1.0 : 0.0, b == 2 ? 1.0 : 0.0};
        pair_accumulate<WALL, double>(d[0], d[1], d[2], ri[2], rj[2], f[0], f[1], f[2], k, u[0],
                                      u[1], u[2]);
        m[b] = u[0];
        m[3 + b] = u[1];
        m[6 + b] = u[2];
    }
}

// ---------------------------------------------------------------------------
// Packed variant: the same pair interaction for two targets at once, one in
// each half of a float2, with Blackwell's paired FP32 instructions
// (fma/add/mul .f32x2).  Every source operand arrives duplicated in both
// halves; positions arrive negated so that separations are sums.
struct PairConsts2 {
    float2 a2, c1, c2, c3, c4, sw, tiny, one;
    float four_a2, k1, k2;
    // wall polynomial coefficients (see the f1..f5 formulas above)
    float2 m1, m2, p2, m2o3, p2o3, m10o3, p6, m10, p70o3, p20, m4, p40o3, m140o3, m12, m20o3,
        m8o3;

    __host__ static PairConsts2 make(double a)
    {
        auto d = [](double v) { return make_float2((float)v, (float)v); };
        PairConsts2 k;
        k.a2 = d(a * a);
        k.c1 = d(0.75 * a);
        k.c2 = d(0.5 * a * a * a);
        k.c3 = d(0.75 * a);
        k.c4 = d(-1.5 * a * a * a);
        k.sw = d(0.75 * a);
        k.tiny = d(1e-30);
        k.one = d(1.0);
        k.four_a2 = (float)(4.0 * a * a);
        k.k1 = (float)(9.0 / (32.0 * a));
        k.k2 = (float)(3.0 / (32.0 * a));
        k.m1 = d(-1.0); k.m2 = d(-2.0); k.p2 = d(2.0);
        k.m2o3 = d(-2.0 / 3.0); k.p2o3 = d(2.0 / 3.0); k.m10o3 = d(-10.0 / 3.0);
        k.p6 = d(6.0); k.m10 = d(-10.0); k.p70o3 = d(70.0 / 3.0); k.p20 = d(20.0);
        k.m4 = d(-4.0); k.p40o3 = d(40.0 / 3.0); k.m140o3 = d(-140.0 / 3.0);
        k.m12 = d(-12.0); k.m20o3 = d(-20.0 / 3.0); k.m8o3 = d(-8.0 / 3.0);
        return k;
    }
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }

// u += M_ij f_j for the two targets held in the halves of the float2s.
// dxy2 must already include the tiny floor (it keeps r^2 > 0 for i = j).
template <bool WALL>
__device__ __forceinline__ void pair_accumulate2(float2 dx, float2 dy, float2 dz, float2 dxy2,
                                                 float2 zt, float2 zj, float2 fx, float2 fy,
                                                 float2 fz, const PairConsts2 &k, float2 &ux,
                                                 float2 &uy, float2 &uz)
{
    const float2 r2 = fma2(dz, dz, dxy2);
    const float2 inv = rsqrt2(r2);
    const float2 inv2 = mul2(inv, inv);
    float2 C = mul2(inv, fma2(k.c2, inv2, k.c1));
    float2 D = mul2(mul2(inv, inv2), fma2(k.c4, inv2, k.c3));
    if (__any_sync(0xffffffffu, (r2.x < k.four_a2) | (r2.y < k.four_a2))) {
        // overlapping blobs (rare): regularised branch, lane by lane
        if (r2.x < k.four_a2) { C.x = 1.f - k.k1 * (r2.x * inv.x); D.x = k.k2 * inv.x; }
        if (r2.y < k.four_a2) { C.y = 1.f - k.k1 * (r2.y * inv.y); D.y = k.k2 * inv.y; }
    }
    const float2 rf_xy = fma2(dx, fx, mul2(dy, fy));
    const float2 g = mul2(D, fma2(dz, fz, rf_xy));
    if (!WALL) {
        ux = fma2(C, fx, fma2(g, dx, ux));
        uy = fma2(C, fy, fma2(g, dy, uy));
        uz = fma2(C, fz, fma2(g, dz, uz));
        return;
    }
    const float2 R3 = add2(zt, zj);
    const float2 invR = rsqrt2(fma2(R3, R3, dxy2));
    const float2 hs = mul2(zj, invR);
    const float2 ht = mul2(zt, invR);
    const float2 e3 = add2(hs, ht);
    const float2 E = mul2(e3, e3);
    const float2 t2 = mul2(k.a2, mul2(invR, invR));
    const float2 t4 = mul2(t2, t2);
    const float2 p = mul2(hs, ht);
    const float2 T1 = mul2(E, t2);
    const float2 T2 = mul2(E, t4);
    const float2 hs2 = add2(hs, hs);
    // f1 = -1 - 2p + 2 T1 - 2/3 t2 + 2/3 t4 - 10/3 T2
    const float2 f1 = fma2(k.m10o3, T2, fma2(k.p2o3, t4, fma2(k.m2o3, t2, fma2(k.p2, T1, fma2(k.m2, p, k.m1)))));
    // f2 = -1 + 6p - 10 T1 + 2 t2 + 70/3 T2 - 10/3 t4
    const float2 f2 = fma2(k.m10o3, t4, fma2(k.p70o3, T2, fma2(k.p2, t2, fma2(k.m10, T1, fma2(k.p6, p, k.m1)))));
    // f3 = 2 hs + e3 (20 T1 - 4 t2 + 40/3 t4 - 140/3 T2 - 12 p)
    const float2 in3 = fma2(k.m12, p, fma2(k.m140o3, T2, fma2(k.p40o3, t4, fma2(k.m4, t2, mul2(k.p20, T1)))));
    const float2 f3 = fma2(e3, in3, hs2);
    // f4 = 2 hs - 20/3 e3 t4
    const float2 f4 = fma2(k.m20o3, mul2(e3, t4), hs2);
    // f5 = -4 (hs^2 + T1) + 20 T2 - 8/3 t4
    const float2 f5 = fma2(k.m4, fma2(hs, hs, T1), fma2(k.p20, T2, mul2(k.m8o3, t4)));
    const float2 eF = mul2(fma2(R3, fz, rf_xy), invR);
    const float2 gw = mul2(fma2(f2, eF, mul2(f3, fz)), invR);
    const float2 kz = fma2(f4, eF, mul2(f5, fz));
    const float2 s = mul2(k.sw, invR);
    const float2 Cx = fma2(s, f1, C);
    const float2 Gx = fma2(s, gw, g);
    ux = fma2(Cx, fx, fma2(Gx, dx, ux));
    uy = fma2(Cx, fy, fma2(Gx, dy, uy));
    uz = fma2(Cx, fz, fma2(g, dz, fma2(s, fma2(gw, R3, kz), uz)));
}

// Both directions of one unordered pair at once (M_ji = M_ij^T): forward
// u_i += M_ij f_j into (ux, uy, uz) and reverse v_j += M_ij^T f_i into
// (rx, ry, rz).  The transpose reuses every coefficient; only
// the roles of f3 and f4 swap.  Packed over two targets i as in
// pair_accumulate2; fi* are the targets' forces.
// FAR: the caller guarantees that no pair is closer than 2a (block pairs
// whose bounding boxes are far apart), so the overlap test is left out.
template <bool WALL, bool FAR = false>
__device__ __forceinline__ void pair_sym2(float2 dx, float2 dy, float2 dz, float2 dxy2, float2 zt,
                                          float2 zj, float2 fx, float2 fy, float2 fz, float2 fix,
                                          float2 fiy, float2 fiz, const PairConsts2 &k, float2 &ux,
                                          float2 &uy, float2 &uz, float2 &rx, float2 &ry,
                                          float2 &rz)
{
    const float2 r2 = fma2(dz, dz, dxy2);
    const float2 inv = rsqrt2(r2);
    const float2 inv2 = mul2(inv, inv);
    float2 C = mul2(inv, fma2(k.c2, inv2, k.c1));
    float2 D = mul2(mul2(inv, inv2), fma2(k.c4, inv2, k.c3));
    if (!FAR && __any_sync(0xffffffffu, (r2.x < k.four_a2) | (r2.y < k.four_a2))) {
        if (r2.x < k.four_a2) { C.x = 1.f - k.k1 * (r2.x * inv.x); D.x = k.k2 * inv.x; }
        if (r2.y < k.four_a2) { C.y = 1.f - k.k1 * (r2.y * inv.y); D.y = k.k2 * inv.y; }
    }
    const float2 rf_xy = fma2(dx, fx, mul2(dy, fy));
    const float2 g = mul2(D, fma2(dz, fz, rf_xy));
    const float2 rb_xy = fma2(dx, fix, mul2(dy, fiy));
    const float2 gb = mul2(D, fma2(dz, fiz, rb_xy));
    if (!WALL) {
        ux = fma2(C, fx, fma2(g, dx, ux));
        uy = fma2(C, fy, fma2(g, dy, uy));
        uz = fma2(C, fz, fma2(g, dz, uz));
        rx = fma2(C, fix, fma2(gb, dx, rx));
        ry = fma2(C, fiy, fma2(gb, dy, ry));
        rz = fma2(C, fiz, fma2(gb, dz, rz));
        return;
    }
    const float2 R3 = add2(zt, zj);
    const float2 invR = rsqrt2(fma2(R3, R3, dxy2));
    const float2 hs = mul2(zj, invR);
    const float2 ht = mul2(zt, invR);
    const float2 e3 = add2(hs, ht);
    const float2 E = mul2(e3, e3);
    const float2 invR2 = mul2(invR, invR);
    const float2 t2 = mul2(k.a2, invR2);
    const float2 t4 = mul2(t2, t2);
    const float2 p = mul2(hs, ht);
    const float2 T1 = mul2(E, t2);
    const float2 T2 = mul2(E, t4);
    const float2 hs2 = add2(hs, hs);
    const float2 f1 = fma2(k.m10o3, T2, fma2(k.p2o3, t4, fma2(k.m2o3, t2, fma2(k.p2, T1, fma2(k.m2, p, k.m1)))));
    const float2 f2 = fma2(k.m10o3, t4, fma2(k.p70o3, T2, fma2(k.p2, t2, fma2(k.m10, T1, fma2(k.p6, p, k.m1)))));
    const float2 in3 = fma2(k.m12, p, fma2(k.m140o3, T2, fma2(k.p40o3, t4, fma2(k.m4, t2, mul2(k.p20, T1)))));
    const float2 f3 = fma2(e3, in3, hs2);
    const float2 f4 = fma2(k.m20o3, mul2(e3, t4), hs2);
    const float2 f5 = fma2(k.m4, fma2(hs, hs, T1), fma2(k.p20, T2, mul2(k.m8o3, t4)));
    const float2 s = mul2(k.sw, invR);
    const float2 Cx = fma2(s, f1, C);
    // With R.f = rf_xy + R3 fz (unnormalised), the forms above read
    // gw = f2 R.f / rho^2 + f3 fz / rho and kz = f4 R.f / rho + f5 fz, so
    // f2 / rho^2, f3 / rho and f4 / rho serve both directions.
    const float2 A2 = mul2(f2, invR2);
    const float2 A3 = mul2(f3, invR);
    const float2 A4 = mul2(f4, invR);
    // forward: M_ij f_j
    const float2 RF = fma2(R3, fz, rf_xy);
    const float2 gw = fma2(A2, RF, mul2(A3, fz));
    const float2 kz = fma2(A4, RF, mul2(f5, fz));
    const float2 Gx = fma2(s, gw, g);
    ux = fma2(Cx, fx, fma2(Gx, dx, ux));
    uy = fma2(Cx, fy, fma2(Gx, dy, uy));
    uz = fma2(Cx, fz, fma2(g, dz, fma2(s, fma2(gw, R3, kz), uz)));
    // reverse: M_ij^T f_i (f3 and f4 exchange roles)
    const float2 RB = fma2(R3, fiz, rb_xy);
    const float2 gwb = fma2(A2, RB, mul2(A4, fiz));
    const float2 kzb = fma2(A3, RB, mul2(f5, fiz));
    const float2 Gb = fma2(s, gwb, gb);
    rx = fma2(Cx, fix, fma2(Gb, dx, rx));
    ry = fma2(Cx, fiy, fma2(Gb, dy, ry));
    rz = fma2(Cx, fiz, fma2(gb, dz, fma2(s, fma2(gwb, R3, kzb), rz)));
}

}  // namespace mb

