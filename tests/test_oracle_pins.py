"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a textbook limit or a number printed in the paper.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PI = math.pi


def _rng(seed=0):
    return np.random.default_rng(seed)


# ------------------------------------------------------------ free-space RPY
def test_single_blob_stokes_drag():
    """P1: M_ii = (6 pi eta a)^-1 I (Section 2.1.1, after Eq. RPYTensor)."""
    for a, eta in [(0.5, 1.0), (0.13, 2.5)]:
        M = O.block([1.0, 2.0, 3.0], [1.0, 2.0, 3.0], a, eta, wall=False)
        np.testing.assert_allclose(M, np.eye(3) / (6 * PI * eta * a), rtol=1e-15, atol=0)


def test_rpy_far_field_is_oseen():
    """P2: for r >> a the RPY tensor tends to the Oseen tensor (Eq. OseenTensor)
    divided by eta, with a relative correction O(a^2/r^2)."""
    rng = _rng(1)
    a, eta = 0.3, 1.7
    for _ in range(5):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        r = 1.0e3 * a
        M = O.block(np.zeros(3), r * d, a, eta, wall=False)
        oseen = (np.eye(3) + np.outer(d, d)) / (8 * PI * eta * r)
        np.testing.assert_allclose(M, oseen, rtol=0, atol=3 * (a / r) ** 2 * np.abs(oseen).max())


def test_rpy_continuous_at_contact():
    """P4: both branches of Eq. RPYTensor meet at r = 2a, with C1 = C3 = 7/16
    and C2 = C4 = 3/16 there."""
    a = 0.7
    d = np.array([0.6, -0.8, 0.0])
    lo = O.block(np.zeros(3), (2 * a) * (1 - 1e-12) * d, a, wall=False)
    hi = O.block(np.zeros(3), (2 * a) * (1 + 1e-12) * d, a, wall=False)
    np.testing.assert_allclose(lo, hi, atol=1e-11 / a)
    expect = (7 / 16 * np.eye(3) + 3 / 16 * np.outer(d, d)) / (6 * PI * a)
    np.testing.assert_allclose(hi, expect, atol=1e-11 / a)


def test_rpy_overlap_branch_limits():
    """Near branch of Eq. RPYTensor: r -> 0 recovers the self mobility, and the
    matrix of two overlapping blobs stays positive definite."""
    a = 1.0
    d = np.array([0.0, 0.0, 1.0])
    M = O.block(np.zeros(3), 1e-9 * d, a, wall=False)
    np.testing.assert_allclose(M, np.eye(3) / (6 * PI * a), atol=1e-9)
    for sep in (0.1, 0.5, 1.0, 1.9):
        r = np.array([[0, 0, 0], [sep, 0.2 * sep, 0]], dtype=float)
        np.linalg.cholesky(O.mobility_matrix(r, a, wall=False))


def test_effective_radii_table():
    """P3: R_h and R_tau of 12/42/162/642-blob shells at a/s = 1/2 and 1/4
    reproduce Table Stresslets_3D (left) to the printed digits."""
    g = json.load(open(os.path.join(GOLDEN, "effective_radii.json")))
    for n, ratio, rh_ref, rt_ref in g["rows"]:
        rho = I.shell(int(n))
        a = ratio * I.min_spacing(rho)
        N = O.body_mobility(rho, np.zeros((1, 3)), np.array([0, n]), a, 1.0, wall=False)
        rh = 1.0 / (6 * PI * np.trace(N[:3, :3]) / 3)
        rt = (1.0 / (8 * PI * np.trace(N[3:, 3:]) / 3)) ** (1 / 3)
        assert abs(rh - rh_ref) <= 1.5e-4, (n, ratio, rh, rh_ref)
        assert abs(rt - rt_ref) <= 1.5e-4, (n, ratio, rt, rt_ref)


# ------------------------------------------------------------ wall correction
def test_wall_green_function_no_slip():
    """Blake's construction: (1 + a^2/6 Lap_y) applied to Oseen + image vanishes
    for every target on the wall z = 0, for any source height and a."""
    rng = _rng(2)
    for _ in range(20):
        y = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), rng.uniform(0.2, 4)])
        x = np.array([rng.uniform(-3, 3), rng.uniform(-3, 3), 0.0])
        a = rng.uniform(0.05, 0.5)
        img, free = O.source_faxen_fields(x, y, a)
        assert np.abs(img + free).max() <= 1e-13 * np.abs(free).max()
        # away from the wall the sum is not zero (the check is not vacuous)
        x[2] = 0.5
        img, free = O.source_faxen_fields(x, y, a)
        assert np.abs(img + free).max() > 1e-3 * np.abs(free).max()


def test_wall_self_mobility_closed_form():
    """P5: self mobility of a blob at height h (in units of a) above the wall:
    parallel 1 - 9/(16h) + 1/(8h^3) - 1/(16h^5), perpendicular
    1 - 9/(8h) + 1/(2h^3) - 1/(8h^5) (Rotne-Prager-Blake; the leading -9/16
    is the fn2 of mu_tt^par in Table FittingSphereWall)."""
    for a in (0.12, 0.5, 1.0):
        for hh in (1.0, 1.3, 2.0, 5.0, 40.0):
            M = O.block([0.4, -0.2, hh * a], [0.4, -0.2, hh * a], a) * 6 * PI * a
            par = 1 - 9 / (16 * hh) + 1 / (8 * hh**3) - 1 / (16 * hh**5)
            perp = 1 - 9 / (8 * hh) + 1 / (2 * hh**3) - 1 / (8 * hh**5)
            np.testing.assert_allclose(np.diag(M), [par, par, perp], rtol=1e-13)
            assert np.abs(M - np.diag(np.diag(M))).max() < 1e-15


def test_wall_mobility_symmetric_positive_definite():
    """P6: M = M^T and Cholesky succeeds for blobs at z in [a, 3a]
    (Section 2.1.1: SPD when no blob overlaps the wall)."""
    rng = _rng(3)
    for trial in range(3):
        a = 0.5
        r = np.column_stack([rng.uniform(0, 6, 40), rng.uniform(0, 6, 40), rng.uniform(a, 3 * a, 40)])
        M = O.mobility_matrix(r, a)
        assert np.abs(M - M.T).max() <= 1e-14 * np.abs(M).max()
        np.linalg.cholesky(M)
        assert np.linalg.eigvalsh(M).min() > 0


def test_wall_correction_vanishes_far_from_wall():
    """P7: far from the wall the correction decays and the free RPY tensor is
    recovered; the self correction approaches -(9/16)(a/h) (parallel)."""
    a = 0.5
    for h in (1e2, 1e3, 1e4):
        W = O.wall_block([0, 0, h], [0, 0, h], a) * 6 * PI * a
        assert abs(W[0, 0] + 9 / 16 * a / h) < 2 * (a / h) ** 3
        assert abs(W[2, 2] + 9 / 8 * a / h) < 2 * (a / h) ** 3
        Wp = O.wall_block([0, 0, h], [1.5, 0.3, h + 0.7], a)
        Mp = O.rpy_free_block([0, 0, h], [1.5, 0.3, h + 0.7], a)
        assert np.abs(Wp).max() < 2 * (3 / h) * np.abs(Mp).max()


def test_sphere_near_wall_matches_paper_fits():
    """P9: 642-blob shell (a = s/2) at heights H/R_h in {1.1, 1.5, 2, 4},
    averaged over orientations, against the fits of Table FittingSphereWall."""
    g = json.load(open(os.path.join(GOLDEN, "sphere_wall_fits.json")))["fits"]

    def fit(key, x):
        d, al, n2, n1, n0, d1, d0, _ = g[key]
        return d + x ** (-al) * (n2 * x * x + n1 * x + n0) / (x * x + d1 * x + d0)

    rho = I.shell(642)
    a = 0.5 * I.min_spacing(rho)
    bs = np.array([0, 642])
    N0 = O.body_mobility(rho, np.zeros((1, 3)), bs, a, 1.0, wall=False)
    Rh = 1 / (6 * PI * np.trace(N0[:3, :3]) / 3)
    Rt = (1 / (8 * PI * np.trace(N0[3:, 3:]) / 3)) ** (1 / 3)
    rng = _rng(4)
    tol = {"tt_parallel": 6e-3, "rr_parallel": 1e-3, "rr_perpendicular": 2e-4, "rt_parallel": 2e-2}
    for x in (1.1, 1.5, 2.0, 4.0):
        q = np.array([[0.0, 0.0, x * Rh]])
        vals = {k: [] for k in tol}
        for th in I.random_unit_quaternions(rng, 3):
            r = O.blob_positions(q, th[None], bs, rho)
            N = O.body_mobility(r, q, bs, a, 1.0, wall=True)
            vals["tt_parallel"].append((N[0, 0] + N[1, 1]) / 2 * 6 * PI * Rh)
            vals["rr_parallel"].append((N[3, 3] + N[4, 4]) / 2 * 8 * PI * Rt**3)
            vals["rr_perpendicular"].append(N[5, 5] * 8 * PI * Rt**3)
            vals["rt_parallel"].append((N[4, 0] - N[3, 1]) / 2 * 6 * PI * Rh**2)
        for k, v in vals.items():
            ref = fit(k, x)
            assert abs(np.mean(v) - ref) <= tol[k] * abs(ref), (k, x, np.mean(v), ref)


# ------------------------------------------------------------ bodies and solve
def test_rotation_matches_library_quaternion():
    """Scalar-first Hamilton convention: the oracle's rotation equals scipy's
    rotation of the same quaternion (scalar-last there), and is proper."""
    rng = _rng(5)
    for th in I.random_unit_quaternions(rng, 10):
        R = O.rotation_matrix(th)
        ref = Rotation.from_quat([th[1], th[2], th[3], th[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-14)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14


def test_K_and_KT_are_adjoint_and_rigid():
    """Eq. noslip_rigid: K U is a rigid velocity field; K^T is its adjoint
    (total force and torque about q_p)."""
    s = I.config_small_suspension(3)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = _rng(6)
    U, W = rng.standard_normal((s.n_bodies, 3)), rng.standard_normal((s.n_bodies, 3))
    lam = rng.standard_normal((s.n_blobs, 3))
    v = O.K_apply(U, W, r, s.q, s.blob_start)
    F, T = O.KT_apply(lam, r, s.q, s.blob_start)
    assert abs(np.sum(v * lam) - (np.sum(U * F) + np.sum(W * T))) < 1e-11 * np.abs(v * lam).sum()
    K = O.K_matrix(r, s.q, s.blob_start)
    np.testing.assert_allclose(K @ np.concatenate([U, W], 1).reshape(-1), v.reshape(-1), atol=1e-13)
    # rigid: pairwise distances are preserved to first order, (v_i - v_j).(r_i - r_j) = 0
    for p in range(s.n_bodies):
        lo = s.blob_start[p]
        for i in range(lo, lo + 5):
            assert abs(np.dot(v[i] - v[lo + 7], r[i] - r[lo + 7])) < 1e-12


def test_dimer_closed_form():
    """P8: two blobs at separation d > 2a in free space.  Force along the axis
    splits evenly, U = (1 + C1 + C2)/(6 pi eta a) F/2; across it,
    U = (1 + C1)/(6 pi eta a) F/2; a torque about a perpendicular axis gives
    omega = 2 (1 - C1) tau / (6 pi eta a d^2)."""
    a, eta, d = 0.4, 1.3, 1.5
    C1 = 3 * a / (4 * d) + a**3 / (2 * d**3)
    C2 = 3 * a / (4 * d) - 3 * a**3 / (2 * d**3)
    rho = np.array([[-d / 2, 0, 0], [d / 2, 0, 0]])
    q = np.array([[0.0, 0.0, 0.0]])
    bs = np.array([0, 2])
    mu = 1 / (6 * PI * eta * a)
    # K^T M^-1 K is singular for a dimer (it cannot spin about its axis), so the
    # saddle system is solved in the least-squares (pseudo-inverse) sense.
    def solver(*args, **kw):
        return O.solve_saddle(*args, pinv=True, **kw)

    U, W, lam = solver(rho, q, bs, np.array([[1.0, 0, 0]]), np.array([[0, 0, 0.0]]), a, eta, wall=False)
    np.testing.assert_allclose(U[0], [mu * (1 + C1 + C2) / 2, 0, 0], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(lam, [[0.5, 0, 0], [0.5, 0, 0]], atol=1e-12)
    U, W, lam = solver(rho, q, bs, np.array([[0, 1.0, 0]]), np.array([[0, 0, 0.0]]), a, eta, wall=False)
    np.testing.assert_allclose(U[0], [0, mu * (1 + C1) / 2, 0], rtol=1e-12, atol=1e-14)
    U, W, lam = solver(rho, q, bs, np.zeros((1, 3)), np.array([[0, 0, 1.0]]), a, eta, wall=False)
    np.testing.assert_allclose(W[0], [0, 0, 2 * (1 - C1) * mu / d**2], rtol=1e-12, atol=1e-14)


def test_direct_and_schur_solves_agree():
    """Eq. saddle_M solved by LU equals Eq. BodyMob solved by Cholesky, and the
    solution satisfies the balance rows exactly."""
    s = I.config_small_suspension(1)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    U1, W1, l1 = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, s.eta)
    U2, W2, l2 = O.solve_schur(r, s.q, s.blob_start, s.F, s.T, s.a, s.eta)
    np.testing.assert_allclose(U1, U2, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(W1, W2, rtol=1e-9, atol=1e-12)
    F, T = O.KT_apply(l1, r, s.q, s.blob_start)
    np.testing.assert_allclose(F, s.F, atol=1e-10)
    np.testing.assert_allclose(T, s.T, atol=1e-10)
    res = O.residual_rows(np.arange(s.n_blobs), r, s.q, s.blob_start, l1, U1, W1, s.a, s.eta)
    assert np.abs(res).max() < 1e-10 * np.abs(U1).max()


def test_preconditioner_is_exact_for_one_body():
    """Eq. indef_block_P: for a single body the block-diagonal mobility is the
    full mobility, so applying the preconditioner solves Eq. saddle_M."""
    s = I.sphere_suspension(7, 1, 42, 0.243, 4.0, 1.5, 2.0)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    U, W, lam = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a)
    lam_p, UW = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, np.zeros((42, 3)),
                                -np.concatenate([s.F, s.T], 1))
    np.testing.assert_allclose(lam_p, lam, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(UW[0, :3], U[0], rtol=1e-9)
    np.testing.assert_allclose(UW[0, 3:], W[0], rtol=1e-9)


def test_matvec_equals_dense_product():
    """The double-loop matvec and the assembled matrix give the same product
    (including a target subset)."""
    r, f = I.blob_cloud(8, 200, 0.5, 8.0, 0.5, 1.5)
    M = O.mobility_matrix(r, 0.5)
    u = O.matvec(r, f, 0.5)
    np.testing.assert_allclose(u.reshape(-1), M @ f.reshape(-1), rtol=1e-13, atol=1e-15)
    t = np.array([5, 0, 199, 17])
    np.testing.assert_allclose(O.matvec(r, f, 0.5, targets=t), u[t], rtol=1e-14)


# ------------------------------------------------------------ resistance problem
def test_resistance_of_isotropic_shell_matches_effective_radii():
    """Eq. resistance_problem for one 12-blob shell in an unbounded domain:
    the icosahedral symmetry makes its resistance isotropic, so translating
    at U needs F = 6 pi eta R_h U and rotating at Omega needs
    T = 8 pi eta R_tau^3 Omega, with R_h and R_tau of Table Stresslets_3D."""
    g = json.load(open(os.path.join(GOLDEN, "effective_radii.json")))
    for n, ratio, rh_ref, rt_ref in g["rows"]:
        if n != 12:
            continue
        rho = I.shell(12)
        a = ratio * I.min_spacing(rho)
        q = np.zeros((1, 3))
        for axis in range(3):
            e = np.zeros((1, 3))
            e[0, axis] = 1.0
            F, T, _ = O.solve_resistance(rho, q, np.array([0, 12]), e, np.zeros((1, 3)), a, 1.0,
                                         wall=False)
            assert abs(F[0, axis] / (6 * PI) - rh_ref) <= 1.5e-4
            assert np.abs(np.delete(F[0], axis)).max() <= 1e-12 and np.abs(T).max() <= 1e-12
            F, T, _ = O.solve_resistance(rho, q, np.array([0, 12]), np.zeros((1, 3)), e, a, 1.0,
                                         wall=False)
            assert abs((T[0, axis] / (8 * PI)) ** (1 / 3) - rt_ref) <= 1.5e-4
            assert np.abs(np.delete(T[0], axis)).max() <= 1e-12 and np.abs(F).max() <= 1e-12


def test_resistance_inverts_the_mobility_problem():
    """Section 2.1.2: the body resistance R = K^T M^-1 K is the inverse of the
    body mobility N.  Solving the mobility problem for (U, Omega) under given
    (F, T) and slip, then the resistance problem with that motion and slip,
    returns the forces and torques and the same blob forces."""
    s = I.mixed_suspension(11, 4)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    slip = _rng(3).standard_normal((s.n_blobs, 3)) * 0.2
    U, W, lam = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, 1.0, True, slip)
    F, T, lam2 = O.solve_resistance(r, s.q, s.blob_start, U, W, s.a, 1.0, True, slip)
    np.testing.assert_allclose(F, s.F, rtol=0, atol=1e-9 * np.abs(s.F).max())
    np.testing.assert_allclose(T, s.T, rtol=0, atol=1e-9 * np.abs(s.F).max())
    np.testing.assert_allclose(lam2, lam, rtol=0, atol=1e-9 * np.abs(lam).max())


def test_resistance_rigid_slip_cancels_motion():
    """A slip equal to minus a rigid motion of the bodies, with the bodies
    moving by that motion, leaves the fluid at rest: lambda = 0, F = T = 0."""
    s = I.config_small_suspension(2)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = _rng(4)
    V, Wv = rng.standard_normal((s.n_bodies, 3)), rng.standard_normal((s.n_bodies, 3))
    slip = -O.K_apply(V, Wv, r, s.q, s.blob_start)
    F, T, lam = O.solve_resistance(r, s.q, s.blob_start, V, Wv, s.a, 1.0, True, slip)
    assert np.abs(lam).max() <= 1e-12 and np.abs(F).max() <= 1e-12 and np.abs(T).max() <= 1e-12


# ------------------------------------------------------------ active slip
def _strain_slip(rho, gamma=1.0):
    """Apparent slip -v(r_i) for the planar strain v = gamma (x, -y, 0)."""
    return -gamma * np.stack([rho[:, 0], -rho[:, 1], np.zeros(len(rho))], axis=1)


def _stresslet_11(lam, rho):
    """s_11 of the symmetric traceless first moment sum_i lambda_i (x) r_i."""
    S = lam.T @ rho
    s = 0.5 * (S + S.T) - np.trace(S) / 3.0 * np.eye(3)
    return s[0, 0]


def test_stresslet_radii_table():
    """R_s of force- and torque-free shells under the strain slip reproduces
    Table Stresslets_3D (left); the free body does not move."""
    g = json.load(open(os.path.join(GOLDEN, "stresslet_radii.json")))
    for n, ratio, rs_ref in g["rows"]:
        rho = I.shell(int(n))
        a = ratio * I.min_spacing(rho)
        z = np.zeros((1, 3))
        U, W, lam = O.solve_saddle(rho, z, np.array([0, n]), z, z, a, 1.0, False,
                                   _strain_slip(rho))
        rs = (-3.0 * _stresslet_11(lam, rho) / (20.0 * PI)) ** (1.0 / 3.0)
        assert abs(rs - rs_ref) <= 1.5e-4, (n, ratio, rs, rs_ref)
        assert np.abs(U).max() <= 1e-12 and np.abs(W).max() <= 1e-12


def squirmer_slip(rho, B1=1.0):
    """Tangential slip B1 sin(theta) e_theta of a squirmer (Section 4.3)."""
    th = np.arccos(np.clip(rho[:, 2] / np.linalg.norm(rho, axis=1), -1.0, 1.0))
    ph = np.arctan2(rho[:, 1], rho[:, 0])
    e_th = np.stack([np.cos(th) * np.cos(ph), np.cos(th) * np.sin(ph), -np.sin(th)], axis=1)
    return B1 * np.sin(th)[:, None] * e_th


def test_squirmer_speed_converges_linearly_in_blob_radius():
    """Section 4.3: a force- and torque-free squirmer swims along z, and the
    relative error of its speed against (2/3) B1 is linear in a/R_g: halving
    a (162 -> 642 blobs at fixed a/s) halves it, and it vanishes with a."""
    eps = []
    for n in (162, 642):
        rho = I.shell(n)
        a = 0.5 * I.min_spacing(rho)
        z = np.zeros((1, 3))
        U, W, _ = O.solve_saddle(rho, z, np.array([0, n]), z, z, a, 1.0, False, squirmer_slip(rho))
        assert np.abs(U[0, :2]).max() <= 1e-12 and np.abs(W).max() <= 1e-12
        eps.append((U[0, 2] / (2.0 / 3.0) - 1.0, a))
    (e1, a1), (e2, a2) = eps
    assert 0 < e2 < e1
    assert abs((e2 / a2) / (e1 / a1) - 1.0) <= 0.05   # the same slope: linear in a


# ------------------------------------------------------------ flow evaluation (Appendix B)
def test_eval_far_field_is_oseen():
    """Far from a blob the velocity of a tracer blob is the Oseen tensor of
    the force, (8 pi eta d)^-1 (I + d d^T / d^2) f, up to O(a^2/d^2)."""
    rng = _rng(9)
    a, eta = 0.3, 1.7
    r = rng.uniform(-1, 1, (1, 3))
    f = rng.standard_normal((1, 3))
    for _ in range(5):
        e = rng.standard_normal(3)
        e /= np.linalg.norm(e)
        d = 3000 * a
        x = r + d * e
        u = O.eval_points(x, r, f, a, eta, wall=False)[0]
        ref = (np.eye(3) + np.outer(e, e)) @ f[0] / (8 * PI * eta * d)
        assert np.abs(u - ref).max() <= 1e-6 * np.abs(ref).max()


def test_render_flow_limits():
    """Appendix B rendering: (1) one sub-blob at the centre with the blob's
    own radius reproduces the blob velocities M lambda; (2) far away the
    rendered flow is the Oseen field of the total force, whatever the split."""
    s = I.config_small_suspension(1)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    lam = _rng(4).standard_normal((s.n_blobs, 3))
    v = O.render_flow(r[:7], r, lam, np.zeros((1, 3)), s.a, 1.0, True)
    np.testing.assert_allclose(v, O.matvec(r, lam, s.a, 1.0, True, targets=np.arange(7)),
                               rtol=1e-13, atol=1e-13)
    rho12 = I.shell(12) * s.a
    one = r[:1]
    F = lam[:1]
    far = one + np.array([[800.0, -300.0, 500.0]])
    v1 = O.render_flow(far, one, F, rho12, 0.05 * s.a, 1.0, False)[0]
    d = far[0] - one[0]
    dn = np.linalg.norm(d)
    ref = (np.eye(3) + np.outer(d, d) / dn ** 2) @ F[0] / (8 * PI * dn)
    assert np.abs(v1 - ref).max() <= 1e-6 * np.abs(ref).max()


# ------------------------------------------------------------ permeable bodies (Appendix C)
def test_permeable_body_darcy_limit():
    """Eq. permeable_slip: with a large shift d = kappa / (eta dV) on every
    blob the body is nearly transparent, lambda ~ K U / d, and the force
    balance K^T lambda = F gives U -> d F / N_b (the translational block of
    K^T K is N_b I when the blobs are centred on the tracking point).  The
    relative deviation is of order N_b times the body's mobility scale
    1/(6 pi eta R_g) over d, and falls like 1/d."""
    rho = I.shell(42)
    a = 0.5 * I.min_spacing(rho)
    F = np.array([[0.3, -1.1, 0.7]])
    z = np.zeros((1, 3))
    dev_prev = None
    for d in (1e3, 1e5):
        U, W, _ = O.solve_saddle(rho, z, np.array([0, 42]), F, z, a, 1.0, False,
                                 shift=np.full(42, d))
        dev = np.linalg.norm(U[0] * 42 / d - F[0]) / np.linalg.norm(F[0])
        assert dev <= 1.5 * 42 / (6 * PI * d)
        if dev_prev is not None:
            assert dev <= dev_prev * 0.02   # ~1/d decay (100x in d)
        dev_prev = dev
        assert np.abs(W).max() <= 1e-9 * np.abs(U).max()


def test_residual_rows_vanish_at_the_direct_solution():
    """The sampled rows of Eq. saddle_M's first block row (evaluated with the
    pair loop, not the dense matrix) vanish at the dense direct solution and
    not at a perturbed one."""
    s = I.config_small_suspension(4)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    U, W, lam = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, 1.0, True)
    rows = np.arange(0, s.n_blobs, 7)
    res = O.residual_rows(rows, r, s.q, s.blob_start, lam, U, W, s.a)
    assert np.abs(res).max() <= 1e-12 * np.abs(lam).max()
    lam2 = lam.copy()
    lam2[rows[3]] += 1e-6 * np.abs(lam).max()
    res2 = O.residual_rows(rows, r, s.q, s.blob_start, lam2, U, W, s.a)
    assert np.abs(res2).max() > 1e-9 * np.abs(lam).max()
