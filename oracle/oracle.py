"""Plain FP64 CPU oracle of the rigid multiblob mobility problem.

ORACLE — TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline leg of bench.py may import this module.  It shares no code with
the CUDA path and never imports it.  Everything is FP64, dense and direct;
the pair loop and the 3x3 blocks live in mb_oracle.c (plain C), the rest is
numpy.

Functions and the passages they follow:
  rotation_matrix, blob_positions   body geometry r_i = q_p + R(theta_p) rho_i
                                    (Section 2.1 notation: tracking point q_p,
                                    orientation quaternion theta_p; the paper
                                    does not fix a quaternion convention; this
                                    oracle uses scalar-first Hamilton)
  block, mobility_matrix, matvec    Eq. RPYTensor plus the single-wall
                                    correction of Section 2.1.1
  K_matrix, K_apply, KT_apply       Eq. noslip_rigid and the force/torque
                                    balance rows of Eq. rigidSystem
  saddle_matrix, solve_saddle       Eq. saddle_M solved directly (LU); the
                                    permeable-body diagonal of Eq.
                                    permeable_slip (Appendix C) as an option
  solve_schur                       Eq. BodyMob: U = N (F - K^T M^-1 slip),
                                    lambda = M^-1 (K U + slip), by Cholesky
  precond_apply                     Eq. saddle_M_precon with the block-diagonal
                                    mobility of Eq. M_tilde_block_diag, one
                                    body at a time, solved directly (LU)
  eval_points, render_flow           velocity of tracer blobs at arbitrary points
                                    (Eq. RPYTensor + wall), and the flow
                                    rendering of Appendix B (blobs split into
                                    smaller blobs sharing their force)
  solve_resistance                  Eq. resistance_problem: M lambda = K U + slip
                                    by Cholesky, then (F, T) = K^T lambda
                                    (Section 2.1.2)
  residual_rows                     rows of Eq. saddle_M's residual for chosen
                                    blobs, for sampled checks at large N
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(HERE, "_build")
_SO = os.path.join(_BUILD, "libmb_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile mb_oracle.c into oracle/_build/libmb_oracle.so (gcc, OpenMP)."""
    src = os.path.join(HERE, "mb_oracle.c")
    hdr = os.path.join(HERE, "wall_blake_faxen.h")
    if (
        not force
        and os.path.exists(_SO)
        and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))
    ):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def load(path: str):
    """ctypes handle of an oracle library built from mb_oracle.c at `path`,
    with the signatures of its entry points."""
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    L.mbo_rpy_free.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
    L.mbo_wall.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, dp]
    L.mbo_block.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
    L.mbo_src_faxen_fields.argtypes = [dp, dp, ctypes.c_double, dp, dp]
    L.mbo_matvec.argtypes = [
        dp, dp, i64, ctypes.POINTER(ctypes.c_int64), i64,
        ctypes.c_double, ctypes.c_double, ctypes.c_int, dp,
    ]
    L.mbo_assemble.argtypes = [dp, i64, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]
    L.mbo_num_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_SO)
    return _lib


def _p(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def num_threads() -> int:
    return int(lib().mbo_num_threads())


# ---------------------------------------------------------------- 3x3 blocks
def rpy_free_block(ri, rj, a, eta=1.0):
    out = np.zeros(9)
    lib().mbo_rpy_free(_p(_c(ri)), _p(_c(rj)), a, eta, _p(out))
    return out.reshape(3, 3)


def wall_block(ri, rj, a, eta=1.0):
    out = np.zeros(9)
    lib().mbo_wall(_p(_c(ri)), _p(_c(rj)), a, eta, _p(out))
    return out.reshape(3, 3)


def block(ri, rj, a, eta=1.0, wall=True):
    out = np.zeros(9)
    lib().mbo_block(_p(_c(ri)), _p(_c(rj)), a, eta, int(bool(wall)), _p(out))
    return out.reshape(3, 3)


def source_faxen_fields(x, y, a):
    """((1 + a^2/6 Lap_y) G_img, (1 + a^2/6 Lap_y) Oseen) at x for a force at y."""
    img = np.zeros(9)
    free = np.zeros(9)
    lib().mbo_src_faxen_fields(_p(_c(x)), _p(_c(y)), a, _p(img), _p(free))
    return img.reshape(3, 3), free.reshape(3, 3)


# ---------------------------------------------------------------- mobility
def mobility_matrix(r, a, eta=1.0, wall=True):
    r = _c(r)
    n = r.shape[0]
    M = np.zeros((3 * n, 3 * n))
    lib().mbo_assemble(_p(r), n, a, eta, int(bool(wall)), _p(M))
    return M


def matvec(r, f, a, eta=1.0, wall=True, targets=None):
    """u_i = sum_j M_ij f_j, FP64 double loop; u for `targets` only if given."""
    r = _c(r)
    f = _c(f)
    n = r.shape[0]
    if targets is None:
        u = np.zeros((n, 3))
        lib().mbo_matvec(_p(r), _p(f), n, None, n, a, eta, int(bool(wall)), _p(u))
    else:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        u = np.zeros((t.shape[0], 3))
        lib().mbo_matvec(
            _p(r), _p(f), n, t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            t.shape[0], a, eta, int(bool(wall)), _p(u),
        )
    return u


# ---------------------------------------------------------------- bodies
def eval_points(x, r, f, a, eta=1.0, wall=True):
    """u(x_t) = sum_j M(x_t, r_j) f_j with the points x as tracer blobs of
    radius a: the matvec over the blobs and the (force-free) points, read at
    the points."""
    x, r, f = _c(x), _c(r), _c(f)
    allr = np.concatenate([r, x])
    allf = np.concatenate([f, np.zeros_like(x)])
    return matvec(allr, allf, a, eta, wall, targets=np.arange(len(r), len(r) + len(x)))


def render_flow(x, r, lam, offsets, a_sub, eta=1.0, wall=True):
    """Appendix B: blob i becomes blobs of radius a_sub at r_i + offsets[k],
    each with lambda_i / len(offsets); the flow at x is that of a tracer blob
    of radius a_sub."""
    r, lam, offsets = _c(r), _c(lam), _c(offsets)
    rs = (r[:, None, :] + offsets[None, :, :]).reshape(-1, 3)
    ls = np.repeat(lam / len(offsets), len(offsets), axis=0)
    return eval_points(x, rs, ls, a_sub, eta, wall)


def rotation_matrix(theta):
    """Rotation of a unit quaternion theta = (s, v), scalar first:
    R = (s^2 - v.v) I + 2 v v^T + 2 s [v]_x ."""
    s = float(theta[0])
    v = np.asarray(theta[1:4], dtype=np.float64)
    vx = np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])
    return (s * s - v @ v) * np.eye(3) + 2.0 * np.outer(v, v) + 2.0 * s * vx


def blob_positions(q, theta, blob_start, rho):
    r = np.zeros_like(np.asarray(rho, dtype=np.float64))
    for p in range(q.shape[0]):
        lo, hi = int(blob_start[p]), int(blob_start[p + 1])
        R = rotation_matrix(theta[p])
        for i in range(lo, hi):
            r[i] = q[p] + R @ rho[i]
    return r


def _cross_matrix(d):
    return np.array([[0.0, -d[2], d[1]], [d[2], 0.0, -d[0]], [-d[1], d[0], 0.0]])


def K_matrix(r, q, blob_start):
    """Dense K (3N x 6 n_b): blob i of body p moves with u_p + w_p x (r_i - q_p)."""
    n = r.shape[0]
    nb = q.shape[0]
    K = np.zeros((3 * n, 6 * nb))
    for p in range(nb):
        for i in range(int(blob_start[p]), int(blob_start[p + 1])):
            d = r[i] - q[p]
            K[3 * i:3 * i + 3, 6 * p:6 * p + 3] = np.eye(3)
            K[3 * i:3 * i + 3, 6 * p + 3:6 * p + 6] = -_cross_matrix(d)
    return K


def K_apply(U, Omega, r, q, blob_start):
    out = np.zeros_like(r)
    for p in range(q.shape[0]):
        for i in range(int(blob_start[p]), int(blob_start[p + 1])):
            out[i] = U[p] + np.cross(Omega[p], r[i] - q[p])
    return out


def KT_apply(lam, r, q, blob_start):
    """K^T lambda = (sum lambda_i, sum (r_i - q_p) x lambda_i) per body."""
    nb = q.shape[0]
    F = np.zeros((nb, 3))
    T = np.zeros((nb, 3))
    for p in range(nb):
        for i in range(int(blob_start[p]), int(blob_start[p + 1])):
            F[p] += lam[i]
            T[p] += np.cross(r[i] - q[p], lam[i])
    return F, T


def _body_vec(F, T):
    return np.concatenate([F, T], axis=1).reshape(-1)


def saddle_matrix(r, q, blob_start, a, eta=1.0, wall=True, shift=None):
    """[[M, -K], [-K^T, 0]] of Eq. saddle_M.  shift (N values or None) adds
    kappa_p / (eta dV_i) to the diagonal of M for the blobs of permeable
    bodies (Eq. permeable_slip, Appendix C)."""
    M = mobility_matrix(r, a, eta, wall)
    if shift is not None:
        M = M + np.diag(np.repeat(_c(shift).reshape(-1), 3))
    K = K_matrix(r, q, blob_start)
    nb6 = K.shape[1]
    return np.block([[M, -K], [-K.T, np.zeros((nb6, nb6))]])


def solve_saddle(r, q, blob_start, F, T, a, eta=1.0, wall=True, slip=None, pinv=False,
                 shift=None):
    """Direct LU solve of Eq. saddle_M; returns (U, Omega, lambda).

    pinv=True takes the minimum-norm least-squares solution instead, the
    pseudo-inverse reading of Section 2.1.2 for bodies whose K^T M^-1 K is
    singular (e.g. blobs on a line cannot spin about it)."""
    n = r.shape[0]
    nb = q.shape[0]
    A = saddle_matrix(r, q, blob_start, a, eta, wall, shift)
    s = np.zeros(3 * n) if slip is None else _c(slip).reshape(-1)
    b = np.concatenate([s, -_body_vec(F, T)])
    x = np.linalg.lstsq(A, b, rcond=1e-12)[0] if pinv else np.linalg.solve(A, b)
    lam = x[: 3 * n].reshape(n, 3)
    UO = x[3 * n:].reshape(nb, 6)
    return UO[:, :3].copy(), UO[:, 3:].copy(), lam


def solve_schur(r, q, blob_start, F, T, a, eta=1.0, wall=True, slip=None):
    """Eq. BodyMob by Cholesky: S = K^T M^-1 K, U = S^-1 (F - K^T M^-1 slip),
    lambda = M^-1 (K U + slip).  Raises numpy.linalg.LinAlgError if M or S is
    not positive definite."""
    import scipy.linalg as sl

    n = r.shape[0]
    nb = q.shape[0]
    M = mobility_matrix(r, a, eta, wall)
    K = K_matrix(r, q, blob_start)
    cM = sl.cho_factor(M, lower=True)
    MiK = sl.cho_solve(cM, K)
    S = K.T @ MiK
    s = np.zeros(3 * n) if slip is None else _c(slip).reshape(-1)
    rhs = _body_vec(F, T) - K.T @ sl.cho_solve(cM, s)
    UO = sl.cho_solve(sl.cho_factor(S, lower=True), rhs)
    lam = sl.cho_solve(cM, K @ UO + s)
    UO = UO.reshape(nb, 6)
    return UO[:, :3].copy(), UO[:, 3:].copy(), lam.reshape(n, 3)


def solve_resistance(r, q, blob_start, U, Omega, a, eta=1.0, wall=True, slip=None):
    """Eq. resistance_problem: the blob forces lambda with M lambda = K [U; Omega]
    + slip, by Cholesky of the dense M, and the body forces and torques
    (F, T) = K^T lambda they add up to.  Returns (F, T, lambda)."""
    import scipy.linalg as sl

    n = r.shape[0]
    M = mobility_matrix(r, a, eta, wall)
    K = K_matrix(r, q, blob_start)
    s = np.zeros(3 * n) if slip is None else _c(slip).reshape(-1)
    lam = sl.cho_solve(sl.cho_factor(M, lower=True), K @ _body_vec(U, Omega) + s)
    FT = (K.T @ lam).reshape(-1, 6)
    return FT[:, :3].copy(), FT[:, 3:].copy(), lam.reshape(n, 3)


def body_mobility(r, q, blob_start, a, eta=1.0, wall=True):
    """N = (K^T M^-1 K)^-1 (Eq. BodyMob), 6 n_b x 6 n_b."""
    M = mobility_matrix(r, a, eta, wall)
    K = K_matrix(r, q, blob_start)
    S = K.T @ np.linalg.solve(M, K)
    return np.linalg.inv(S)


def precond_apply(r, q, blob_start, a, eta, wall, w, g):
    """Apply the indefinite block-diagonal preconditioner (Eq. indef_block_P):
    solve [[M~, -K], [-K^T, 0]] [lambda; U] = [w; g] with M~ the block-diagonal
    mobility of Eq. M_tilde_block_diag, one body at a time by LU.

    w: (N, 3) blob part, g: (n_b, 6) body part.  Returns (lambda (N,3), U (n_b,6)).
    """
    nb = q.shape[0]
    lam = np.zeros_like(_c(w))
    U = np.zeros((nb, 6))
    for p in range(nb):
        lo, hi = int(blob_start[p]), int(blob_start[p + 1])
        rp = r[lo:hi]
        A = saddle_matrix(rp, q[p:p + 1], np.array([0, hi - lo]), a, eta, wall)
        b = np.concatenate([_c(w[lo:hi]).reshape(-1), _c(g[p])])
        x = np.linalg.solve(A, b)
        lam[lo:hi] = x[: 3 * (hi - lo)].reshape(-1, 3)
        U[p] = x[3 * (hi - lo):]
    return lam, U


def residual_rows(rows, r, q, blob_start, lam, U, Omega, a, eta=1.0, wall=True, slip=None):
    """(M lambda)_i - (K U)_i - slip_i for the blobs in `rows` (Eq. saddle_M,
    first block row), each row by a full FP64 pass over all sources."""
    rows = np.asarray(rows, dtype=np.int64)
    Ml = matvec(r, lam, a, eta, wall, targets=rows)
    body_of = np.searchsorted(blob_start, rows, side="right") - 1
    KU = U[body_of] + np.cross(Omega[body_of], r[rows] - q[body_of])
    s = 0.0 if slip is None else _c(slip)[rows]
    return Ml - KU - s
