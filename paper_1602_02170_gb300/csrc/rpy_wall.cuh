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
        k.tiny = sizeof(T) == 4 ? T(1e-30) : T(1e-300);
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

}  // namespace mb
