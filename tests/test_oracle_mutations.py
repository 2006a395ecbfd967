"""The oracle's pins catch plausible mistakes.

Each case plants one mistake of the kind a transcription of the paper could
make: a dropped term, a wrong sign, a wrong index, a transposed operand, a
wrong coefficient.  The mistake goes into a copy of the oracle, never into
the oracle's own files:
- for the blob mobility, a copy of mb_oracle.c and of its generated wall
  header, edited as text, compiled with gcc into a temporary directory and
  swapped in for the oracle's library;
- for the Python parts, the oracle function replaced by a wrong version
  (monkeypatch).
Then the pins of test_oracle_pins.py run in turn, and at least one of them
must fail.  A mistake that every pin let through would mean that the pins
cannot tell that piece of the oracle from a wrong one.
"""
import os
import subprocess

import numpy as np
import pytest

import test_oracle_pins as P
from oracle import oracle as O

ODIR = os.path.dirname(os.path.abspath(O.__file__))

# Every pin, cheap ones first; the 642-blob sphere-near-wall fits come last.
PINS = sorted((getattr(P, k) for k in dir(P) if k.startswith("test_")),
              key=lambda f: (f.__name__ == "test_sphere_near_wall_matches_paper_fits",
                             f.__code__.co_firstlineno))


def _first_failing_pin():
    """Name of the first pin that fails, or None if all pass."""
    for pin in PINS:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError, ValueError):
            return pin.__name__
    return None


def test_pins_pass_on_the_oracle_itself():
    assert _first_failing_pin() is None


# (label, file, original text, replacement): each original occurs exactly once
C_MUTANTS = [
    ("far-field C2: sign of the a^3 term", "mb_oracle.c",
     "cr = 3.0 * a / (4.0 * r) - 3.0 * a * a * a / (2.0 * r * r * r);",
     "cr = 3.0 * a / (4.0 * r) + 3.0 * a * a * a / (2.0 * r * r * r);"),
    ("far-field C1: a^3 term dropped", "mb_oracle.c",
     "ci = 3.0 * a / (4.0 * r) + a * a * a / (2.0 * r * r * r);",
     "ci = 3.0 * a / (4.0 * r);"),
    ("overlap C3: 9/16 for 9/32", "mb_oracle.c",
     "ci = 1.0 - 9.0 * r / (32.0 * a);", "ci = 1.0 - 9.0 * r / (16.0 * a);"),
    ("overlap C4: 3/16 for 3/32", "mb_oracle.c",
     "cr = 3.0 * r / (32.0 * a);", "cr = 3.0 * r / (16.0 * a);"),
    ("branch switch at r = a", "mb_oracle.c", "if (r > 2.0 * a) {", "if (r > a) {"),
    ("separation index typo", "mb_oracle.c", "ri[2] - rj[2]", "ri[2] - rj[1]"),
    ("wall correction with the wrong sign", "mb_oracle.c",
     "out[k] = g[k] / (8.0 * MBO_PI * eta);", "out[k] = -g[k] / (8.0 * MBO_PI * eta);"),
    ("wall prefactor 1/(6 pi eta)", "mb_oracle.c",
     "out[k] = g[k] / (8.0 * MBO_PI * eta);", "out[k] = g[k] / (6.0 * MBO_PI * eta);"),
    ("wall block transposed", "mb_oracle.c",
     "out[k] = g[k] / (8.0 * MBO_PI * eta);",
     "out[k] = g[3 * (k % 3) + k / 3] / (8.0 * MBO_PI * eta);"),
    ("wall correction left out", "mb_oracle.c", "    if (wall) {\n        double w[9];",
     "    if (0) {\n        double w[9];"),
    ("matvec applies the transposed block", "mb_oracle.c",
     "acc[al] += m[3 * al] * f[3 * j] + m[3 * al + 1] * f[3 * j + 1] +\n"
     "                           m[3 * al + 2] * f[3 * j + 2];",
     "acc[al] += m[al] * f[3 * j] + m[3 + al] * f[3 * j + 1] +\n"
     "                           m[6 + al] * f[3 * j + 2];"),
    ("image point not reflected", "wall_blake_faxen.h",
     "const double t4 = x3 + y3;", "const double t4 = x3 - y3;"),
    ("Faxen coefficient a^2/3 for a^2/6", "wall_blake_faxen.h",
     "const double t15 = pow(a, 2);", "const double t15 = 2*pow(a, 2);"),
]


def _mutant_library(tmp_path, fname, old, new):
    texts = {}
    for f in ("mb_oracle.c", "wall_blake_faxen.h"):
        with open(os.path.join(ODIR, f)) as fh:
            texts[f] = fh.read()
    assert texts[fname].count(old) == 1, f"mutation target not unique in {fname}: {old!r}"
    texts[fname] = texts[fname].replace(old, new)
    for f, t in texts.items():
        with open(os.path.join(tmp_path, f), "w") as fh:
            fh.write(t)
    so = os.path.join(tmp_path, "libmutant.so")
    cmd = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-fopenmp",
           os.path.join(tmp_path, "mb_oracle.c"), "-o", so, "-lm"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:  # no OpenMP runtime: the loops run serially
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True)
    return O.load(so)


@pytest.mark.parametrize("label,fname,old,new", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_a_pin_catches_blob_mobility_mistake(tmp_path, monkeypatch, label, fname, old, new):
    monkeypatch.setattr(O, "_lib", _mutant_library(str(tmp_path), fname, old, new))
    assert _first_failing_pin() is not None, f"no pin caught: {label}"


# ----------------------------------------------------------- Python parts
def _rotation_transposed(orig):
    return lambda theta: orig(theta).T


def _rotation_vv_unscaled(orig):
    def R(theta):
        s, v = float(theta[0]), np.asarray(theta[1:4], dtype=np.float64)
        vx = np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])
        return (s * s - v @ v) * np.eye(3) + np.outer(v, v) + 2.0 * s * vx
    return R


def _K_rotation_sign(orig):
    def K(r, q, blob_start):
        out = orig(r, q, blob_start)
        for p in range(q.shape[0]):
            out[:, 6 * p + 3:6 * p + 6] *= -1.0
        return out
    return K


def _K_apply_cross_swapped(orig):
    def K_apply(U, Omega, r, q, blob_start):
        out = np.zeros_like(r)
        for p in range(q.shape[0]):
            for i in range(int(blob_start[p]), int(blob_start[p + 1])):
                out[i] = U[p] + np.cross(r[i] - q[p], Omega[p])
        return out
    return K_apply


def _KT_apply_cross_swapped(orig):
    def KT_apply(lam, r, q, blob_start):
        F, T = orig(lam, r, q, blob_start)
        return F, -T
    return KT_apply


def _KT_apply_about_origin(orig):
    def KT_apply(lam, r, q, blob_start):
        return orig(lam, r, np.zeros_like(q), blob_start)
    return KT_apply


def _saddle_K_sign(orig):
    def saddle_matrix(r, q, blob_start, a, eta=1.0, wall=True, shift=None):
        A = orig(r, q, blob_start, a, eta, wall, shift)
        n3 = 3 * r.shape[0]
        A[:n3, n3:] *= -1.0
        return A
    return saddle_matrix


def _precond_force_sign(orig):
    def precond_apply(r, q, blob_start, a, eta, wall, w, g):
        return orig(r, q, blob_start, a, eta, wall, w, -np.asarray(g))
    return precond_apply


def _precond_without_wall(orig):
    def precond_apply(r, q, blob_start, a, eta, wall, w, g):
        return orig(r, q, blob_start, a, eta, False, w, g)
    return precond_apply


def _resistance_slip_sign(orig):
    def solve_resistance(r, q, blob_start, U, Omega, a, eta=1.0, wall=True, slip=None):
        s = None if slip is None else -np.asarray(slip)
        return orig(r, q, blob_start, U, Omega, a, eta, wall, s)
    return solve_resistance


def _render_force_not_shared(orig):
    def render_flow(x, r, lam, offsets, a_sub, eta=1.0, wall=True):
        return orig(x, r, np.asarray(lam) * len(offsets), offsets, a_sub, eta, wall)
    return render_flow


PY_MUTANTS = [
    ("rotation transposed (R^T for R)", "rotation_matrix", _rotation_transposed),
    ("rotation: v v^T without its factor 2", "rotation_matrix", _rotation_vv_unscaled),
    ("K: Omega x d with the wrong sign", "K_matrix", _K_rotation_sign),
    ("K U: d x Omega for Omega x d", "K_apply", _K_apply_cross_swapped),
    ("K^T: lambda x d for d x lambda", "KT_apply", _KT_apply_cross_swapped),
    ("K^T: torques about the origin, not q_p", "KT_apply", _KT_apply_about_origin),
    ("saddle matrix: +K for -K", "saddle_matrix", _saddle_K_sign),
    ("preconditioner: body rows with the wrong sign", "precond_apply", _precond_force_sign),
    ("preconditioner blocks without the wall", "precond_apply", _precond_without_wall),
    ("resistance: slip with the wrong sign", "solve_resistance", _resistance_slip_sign),
    ("rendering: sub-blobs each carry the whole force", "render_flow", _render_force_not_shared),
]


@pytest.mark.parametrize("label,name,make", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_a_pin_catches_python_oracle_mistake(monkeypatch, label, name, make):
    monkeypatch.setattr(O, name, make(getattr(O, name)))
    assert _first_failing_pin() is not None, f"no pin caught: {label}"
