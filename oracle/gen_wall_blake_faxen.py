"""Write oracle/wall_blake_faxen.h from the definition of the wall correction.

ORACLE TEST INFRASTRUCTURE — run by hand when the definition changes; the
generated header is committed.  Only sympy is used.

What it writes out (Section 2.1.1, Eq. MobilityFaxen, and the single-wall
paragraph that follows Eq. RPYTensor):

  * G(x, y): Blake's Green's function for a point force at y above a no-slip
    wall at z = 0, split as  G = Oseen(x - y) + G_img(x, y), where with
    ybar = (y1, y2, -y3), R = x - ybar, h = y3 and P = diag(1, 1, -1)

      8 pi G_img_ij = -(d_ij/|R| + R_i R_j/|R|^3)
                      + 2 h P_jj d/dR_j [ h R_i/|R|^3 - (d_i3/|R| + R_i R_3/|R|^3) ]

    (i = velocity direction at x, j = force direction at y; h held fixed in
    the R-derivative).  Blake's construction makes G vanish on z = 0.

  * The wall correction of the blob-blob mobility is the image part with the
    Faxen operator applied at both blobs:

      W(x, y) = eta^-1 (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y) G_img(x, y)

    The free-space part of Eq. MobilityFaxen (with its overlap regularisation)
    is the RPY tensor, Eq. RPYTensor, written by hand in mb_oracle.c.

  * For the no-slip pin, the one-sided (source Faxen only) fields
      (1 + a^2/6 Lap_y) G_img(x, y)   and   (1 + a^2/6 Lap_y) Oseen(x - y),
    whose sum must vanish for x on the wall.

The Laplacians are taken with respect to the Cartesian coordinates of x and
of y (h = y3 moves with y), exactly as the definition reads.
"""
import os
import sys

import sympy as sp

HERE = os.path.dirname(os.path.abspath(__file__))


def build():
    x1, x2, x3, y1, y2, y3, a = sp.symbols("x1 x2 x3 y1 y2 y3 a", real=True)
    X = [x1, x2, x3]
    Y = [y1, y2, y3]
    d = lambda i, j: 1 if i == j else 0
    P = [1, 1, -1]
    Rs = sp.symbols("R1 R2 R3", real=True)
    hs = sp.Symbol("h", real=True)
    Rn = sp.sqrt(sum(c**2 for c in Rs))

    def stokeslet(v, vn, i, j):
        return d(i, j) / vn + v[i] * v[j] / vn**3

    def g_img(i, j):  # 8*pi*G_img_ij as a function of R and h
        inner = hs * Rs[i] / Rn**3 - stokeslet(Rs, Rn, i, 2)
        return -stokeslet(Rs, Rn, i, j) + 2 * hs * P[j] * sp.diff(inner, Rs[j])

    to_xy = {Rs[0]: x1 - y1, Rs[1]: x2 - y2, Rs[2]: x3 + y3, hs: y3}
    r = [x1 - y1, x2 - y2, x3 - y3]
    rn = sp.sqrt(sum(c**2 for c in r))
    lap = lambda f, V: sum(sp.diff(f, v, 2) for v in V)
    c = a**2 / 6

    faxen2, src_img, src_free = [], [], []
    for i in range(3):
        for j in range(3):
            g = g_img(i, j).subs(to_xy)
            gy = g + c * lap(g, Y)
            src_img.append(gy)
            faxen2.append(gy + c * lap(gy, X))
            s = stokeslet(r, rn, i, j)
            src_free.append(s + c * lap(s, Y))
    return (x1, x2, x3, y1, y2, y3, a), faxen2, src_img, src_free


def emit(name, args, exprs, doc):
    reps, red = sp.cse(exprs, symbols=sp.numbered_symbols("t"), optimizations="basic")
    lines = [f"/* {doc} */"]
    lines.append(
        f"static void {name}(const double x[3], const double y[3], double a, double out[9])"
    )
    lines.append("{")
    x1, x2, x3, y1, y2, y3, aa = args
    lines.append("    const double x1 = x[0], x2 = x[1], x3 = x[2];")
    lines.append("    const double y1 = y[0], y2 = y[1], y3 = y[2];")
    for s, e in reps:
        lines.append(f"    const double {s} = {sp.ccode(e)};")
    for k, e in enumerate(red):
        lines.append(f"    out[{k}] = {sp.ccode(e)};")
    lines.append("}")
    return "\n".join(lines)


def render() -> str:
    """The header's text, generated from the definition."""
    args, faxen2, src_img, src_free = build()
    parts = [
        "/* GENERATED by oracle/gen_wall_blake_faxen.py from the definition of the\n"
        " * single-wall correction (Section 2.1.1, Eq. MobilityFaxen with Blake's\n"
        " * image system).  Do not edit.  ORACLE TEST INFRASTRUCTURE.\n"
        " * out[3*i + j]: i = velocity component at x, j = force component at y;\n"
        " * every function returns 8*pi times the field for unit viscosity. */",
        "#pragma once",
        "#include <math.h>",
        emit(
            "wall_faxen2_8pi",
            args,
            faxen2,
            "8 pi (1 + a^2/6 Lap_x)(1 + a^2/6 Lap_y) G_img(x, y)",
        ),
        emit(
            "wall_image_src_faxen_8pi",
            args,
            src_img,
            "8 pi (1 + a^2/6 Lap_y) G_img(x, y)",
        ),
        emit(
            "oseen_src_faxen_8pi",
            args,
            src_free,
            "8 pi (1 + a^2/6 Lap_y) Oseen(x - y)",
        ),
    ]
    return "\n\n".join(parts) + "\n"


def main():
    out = os.path.join(HERE, "wall_blake_faxen.h")
    with open(out, "w") as fh:
        fh.write(render())
    print("wrote", out, file=sys.stderr)


if __name__ == "__main__":
    main()
