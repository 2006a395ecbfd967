/*
 * FP64 CPU oracle for the wall-corrected RPY blob mobility.
 *
 * ORACLE — TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code with
 * the CUDA path and is deliberately plain: one 3x3 block at a time, a double
 * loop over blob pairs, no blocking, no reordering.
 *
 * Blob-blob mobility (Section 2.1.1):
 *   M_ij = RPY(r_i - r_j)                 Eq. RPYTensor, written out below
 *        + W(r_i, r_j)   if wall           (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y)
 *                                          applied to the image part of Blake's
 *                                          Green's function (Eq. MobilityFaxen),
 *                                          generated mechanically into
 *                                          wall_blake_faxen.h
 * The wall sits at z = 0 and every blob is expected at z > 0.
 *
 * Layout: positions, forces and velocities are N x 3 row-major doubles;
 * a 3x3 block is row-major with out[3*alpha + beta] = velocity component alpha
 * of blob i per unit force component beta on blob j.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "wall_blake_faxen.h"

#define MBO_PI 3.14159265358979323846

/* Eq. RPYTensor: (6 pi eta a)^-1 [C1 I + C2 rr/r^2] for r > 2a and
 * (6 pi eta a)^-1 [C3 I + C4 rr/r^2] for r <= 2a; r = 0 gives the Stokes
 * self mobility (6 pi eta a)^-1 I. */
void mbo_rpy_free(const double *ri, const double *rj, double a, double eta, double *out)
{
    const double d[3] = {ri[0] - rj[0], ri[1] - rj[1], ri[2] - rj[2]};
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double pref = 1.0 / (6.0 * MBO_PI * eta * a);
    double ci, cr;
    if (r > 2.0 * a) {
        ci = 3.0 * a / (4.0 * r) + a * a * a / (2.0 * r * r * r);
        cr = 3.0 * a / (4.0 * r) - 3.0 * a * a * a / (2.0 * r * r * r);
    } else {
        ci = 1.0 - 9.0 * r / (32.0 * a);
        cr = 3.0 * r / (32.0 * a);
    }
    for (int al = 0; al < 3; ++al)
        for (int be = 0; be < 3; ++be) {
            double e = (al == be) ? ci : 0.0;
            if (r > 0.0)
                e += cr * d[al] * d[be] / (r * r);
            out[3 * al + be] = pref * e;
        }
}

/* Wall correction W(r_i, r_j) = eta^-1 (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y) G_img. */
void mbo_wall(const double *ri, const double *rj, double a, double eta, double *out)
{
    double g[9];
    wall_faxen2_8pi(ri, rj, a, g);
    for (int k = 0; k < 9; ++k)
        out[k] = g[k] / (8.0 * MBO_PI * eta);
}

void mbo_block(const double *ri, const double *rj, double a, double eta, int wall, double *out)
{
    mbo_rpy_free(ri, rj, a, eta, out);
    if (wall) {
        double w[9];
        mbo_wall(ri, rj, a, eta, w);
        for (int k = 0; k < 9; ++k)
            out[k] += w[k];
    }
}

/* One-sided fields for the no-slip check: (1 + a^2/6 Lap_y) applied to the
 * image part and to the Oseen tensor, for unit viscosity, each divided by 8 pi. */
void mbo_src_faxen_fields(const double *x, const double *y, double a, double *img, double *free_)
{
    wall_image_src_faxen_8pi(x, y, a, img);
    oseen_src_faxen_8pi(x, y, a, free_);
    for (int k = 0; k < 9; ++k) {
        img[k] /= 8.0 * MBO_PI;
        free_[k] /= 8.0 * MBO_PI;
    }
}

/* u_i = sum_j M_ij f_j for the targets listed in `targets` (all N if NULL).
 * u has n_targets x 3 entries, in the order of `targets`. */
void mbo_matvec(const double *r, const double *f, int64_t n, const int64_t *targets,
                int64_t n_targets, double a, double eta, int wall, double *u)
{
    if (targets == NULL)
        n_targets = n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n_targets; ++t) {
        const int64_t i = targets ? targets[t] : t;
        double acc[3] = {0.0, 0.0, 0.0};
        double m[9];
        for (int64_t j = 0; j < n; ++j) {
            mbo_block(r + 3 * i, r + 3 * j, a, eta, wall, m);
            for (int al = 0; al < 3; ++al)
                acc[al] += m[3 * al] * f[3 * j] + m[3 * al + 1] * f[3 * j + 1] +
                           m[3 * al + 2] * f[3 * j + 2];
        }
        u[3 * t] = acc[0];
        u[3 * t + 1] = acc[1];
        u[3 * t + 2] = acc[2];
    }
}

/* Dense (3N) x (3N) row-major mobility matrix. */
void mbo_assemble(const double *r, int64_t n, double a, double eta, int wall, double *M)
{
    const int64_t ld = 3 * n;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        double m[9];
        for (int64_t j = 0; j < n; ++j) {
            mbo_block(r + 3 * i, r + 3 * j, a, eta, wall, m);
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be)
                    M[(3 * i + al) * ld + 3 * j + be] = m[3 * al + be];
        }
    }
}

int mbo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
