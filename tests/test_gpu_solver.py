"""Parity of the body kernels, the block-diagonal preconditioner and the
mobility solve with the FP64 oracle.

Bars: blob build, K, K^T and the preconditioner are FP64 throughout (1e-12,
1e-9 for the preconditioner's factorisations); the mobility solve must give
body velocities (U, Omega) within 1e-6 relative of the oracle's direct solve
of Eq. saddle_M, and lambda within 1e-5.
"""
import numpy as np
import pytest
import torch

import paper_1602_02170_gb300 as mb
from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu


def _dev_susp(s):
    return dict(
        q=dev(s.q), theta=dev(s.theta), blob_start=dev(s.blob_start, torch.int64), rho=dev(s.rho),
        F=dev(s.F), T=dev(s.T),
    )


def test_blob_positions(ctx):
    s = I.config_small_suspension(2)
    d = _dev_susp(s)
    got = host(ctx.blob_positions(d["q"], d["theta"], d["blob_start"], d["rho"]))
    ref = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    assert np.abs(got - ref).max() <= 1e-13


def test_blob_positions_mixed_bodies(ctx):
    s = I.mixed_suspension(3, 40)
    d = _dev_susp(s)
    got = host(ctx.blob_positions(d["q"], d["theta"], d["blob_start"], d["rho"]))
    ref = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    assert np.abs(got - ref).max() <= 1e-13


def test_K_and_KT(ctx):
    s = I.mixed_suspension(4, 30)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = np.random.default_rng(1)
    UO = rng.standard_normal((s.n_bodies, 6))
    lam = rng.standard_normal((s.n_blobs, 3))
    d = _dev_susp(s)
    v = host(ctx.K_apply(dev(r), d["q"], d["blob_start"], dev(UO)))
    np.testing.assert_allclose(v, O.K_apply(UO[:, :3], UO[:, 3:], r, s.q, s.blob_start), atol=1e-13)
    FT = host(ctx.KT_apply(dev(r), d["q"], d["blob_start"], dev(lam)))
    F, T = O.KT_apply(lam, r, s.q, s.blob_start)
    np.testing.assert_allclose(FT, np.concatenate([F, T], 1), atol=1e-12)


@pytest.mark.parametrize("wall", [True, False])
def test_preconditioner_apply(ctx, wall):
    """Eq. saddle_M_precon solved per body by the GPU (Cholesky + Schur,
    explicit inverse) equals the oracle's direct LU solve of each body's
    indefinite block."""
    s = I.config_small_suspension(3)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = np.random.default_rng(2)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, wall)
    lam, UO = ctx.precond_apply(dev(w), dev(g))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, wall, w, g)
    assert rel_l2(host(lam), lam_ref) <= 1e-9
    assert rel_l2(host(UO), UO_ref) <= 1e-9


def test_preconditioner_mixed_sizes(ctx):
    """Bodies of different sizes (42-blob shells and 15-blob boomerangs)."""
    s = I.mixed_suspension(6, 12)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = np.random.default_rng(3)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, True)
    lam, UO = ctx.precond_apply(dev(w), dev(g))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, w, g)
    assert rel_l2(host(lam), lam_ref) <= 1e-9
    assert rel_l2(host(UO), UO_ref) <= 1e-9


def test_preconditioner_large_bodies_global_path(ctx):
    """162-blob shells (486 rows) take the factorisation path that keeps the
    Cholesky factor in global memory."""
    s = I.sphere_suspension(5, 3, 162, 0.12, 10.0, 1.2, 1.6)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = np.random.default_rng(4)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, True)
    lam, UO = ctx.precond_apply(dev(w), dev(g))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, w, g)
    assert rel_l2(host(lam), lam_ref) <= 1e-8
    assert rel_l2(host(UO), UO_ref) <= 1e-8


def _many_shells(seed=8, nbod=160):
    # at least as many bodies as the GPU has SMs: one CTA per body (panels of
    # 8 columns in shared memory) instead of a cluster per body; 36 rows per
    # body, so the last panel is ragged
    return I.sphere_suspension(seed, nbod, 12, 0.3, 48.0, 1.5, 4.0)


def test_preconditioner_many_bodies_one_cta_path(ctx):
    """160 12-blob shells: the preconditioner from the one-CTA-per-body
    factorisation equals the oracle's per-body direct solve."""
    s = _many_shells()
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = np.random.default_rng(5)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, True)
    lam, UO = ctx.precond_apply(dev(w), dev(g))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, w, g)
    assert rel_l2(host(lam), lam_ref) <= 1e-9
    assert rel_l2(host(UO), UO_ref) <= 1e-9


def test_preconditioner_many_bodies_singular_block_reported(ctx):
    """The one-CTA path reports an indefinite block (a blob at z = a/2) as
    MB_ESINGULAR naming the body, as the cluster path does."""
    s = _many_shells()
    q = s.q.copy()
    k = 97
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    low = np.argmin(r[s.blob_start[k]:s.blob_start[k + 1], 2]) + s.blob_start[k]
    q[k, 2] -= r[low, 2] - 0.5 * s.a
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    d = _dev_susp(s)
    with pytest.raises(mb.MBError) as ei:
        ctx.precond_setup(dev(r), dev(q), d["blob_start"], s.a, 1.0, True)
    assert ei.value.name == "MB_ESINGULAR"
    assert f"body {k}" in str(ei.value)


def _lattice_bodies(shape, nbod, seed):
    """nbod jittered cubic-lattice bodies of prod(shape) blobs (spacing 2.2 a)."""
    g = np.stack(np.meshgrid(*[np.arange(k) for k in shape], indexing="ij"), -1)
    a = 0.1
    rho1 = (g.reshape(-1, 3) - (np.array(shape) - 1) / 2.0) * (2.2 * a)
    rng = np.random.default_rng(seed)
    nbl = len(rho1)
    rho = np.concatenate([rho1 + 0.01 * a * rng.standard_normal(rho1.shape) for _ in range(nbod)])
    q = np.array([[2.5 * k, 0.3 * k, 1.5 + 0.2 * k] for k in range(nbod)])
    return I.Suspension(q=q, theta=I.random_unit_quaternions(rng, nbod),
                        blob_start=np.arange(nbod + 1, dtype=np.int64) * nbl, rho=rho,
                        F=np.zeros((nbod, 3)), T=np.zeros((nbod, 3)), a=a)


@pytest.mark.parametrize("shape,nbod", [((6, 6, 5), 2), ((10, 10, 7), 1)])
def test_preconditioner_very_large_bodies(ctx, shape, nbod):
    """Bodies of 180 blobs (540 rows) take the split setup with the column of
    L^-1 in shared memory; 700 blobs (2,100 rows) the one-kernel-per-body
    setup."""
    s = _lattice_bodies(shape, nbod, 6)
    rng = np.random.default_rng(7)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    assert r[:, 2].min() > s.a
    w = rng.standard_normal((s.n_blobs, 3))
    gg = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, True)
    lam, UO = ctx.precond_apply(dev(w), dev(gg))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, w, gg)
    assert rel_l2(host(lam), lam_ref) <= 1e-8
    assert rel_l2(host(UO), UO_ref) <= 1e-8


@pytest.mark.parametrize("perturb", [False, True])
def test_shared_free_space_preconditioner_matches_oracle_blocks(ctx, perturb):
    """MB_PRECOND_FREE_SHARED: one factorisation per body shape, applied
    through each body's rotation, equals the oracle's per-body solve with the
    unbounded-domain block (no wall) of every body.  With perturb, one body's
    offsets differ slightly from the other shells of the same blob count, so
    it must get a shape of its own."""
    s = I.mixed_suspension(7, 9)
    rho = s.rho.copy()
    if perturb:
        b0, b1 = s.blob_start[2], s.blob_start[3]
        rho[b0:b1] *= 1.01
    r = O.blob_positions(s.q, s.theta, s.blob_start, rho)
    rng = np.random.default_rng(8)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    ctx.precond_setup_shared(dev(s.theta), dev(s.blob_start, torch.int64), dev(rho), s.a, 1.0)
    lam, UO = ctx.precond_apply(dev(w), dev(g))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, False, w, g)
    assert rel_l2(host(lam), lam_ref) <= 1e-9
    assert rel_l2(host(UO), UO_ref) <= 1e-9


@pytest.mark.parametrize("prec,tol,u_tol", [("fp64", 1e-10, 1e-8), ("mixed", 1e-10, 1e-8)])
def test_solve_with_shared_free_space_preconditioner(ctx, prec, tol, u_tol):
    """The preconditioner changes the iteration count, not the solution: the
    wall suspension solved with the shared unbounded-domain blocks matches the
    oracle's dense direct solve."""
    for s in (I.config_small_suspension(5), I.mixed_suspension(6, 10)):
        d = _dev_susp(s)
        U, W, lam, info = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"],
                                             d["F"], d["T"], s.a, s.eta, True, tol=tol,
                                             maxit=400, restart=100, prec=prec,
                                             precond="free_shared")
        assert info["converged"] == 1
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, s.eta, True)
        assert rel_l2(host(U), Ur) <= u_tol
        assert rel_l2(host(W), Wr) <= 10 * u_tol


def test_preconditioner_singular_block_reported(ctx):
    """A blob at z = a/2 makes its body's wall-corrected block indefinite: the
    setup reports MB_ESINGULAR instead of producing NaNs."""
    s = I.config_small_suspension(1)
    q = s.q.copy()
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    low = np.argmin(r[s.blob_start[2]:s.blob_start[3], 2]) + s.blob_start[2]
    q[2, 2] -= r[low, 2] - 0.5 * s.a  # lowest blob of body 2 to z = a/2
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    d = _dev_susp(s)
    with pytest.raises(mb.MBError) as ei:
        ctx.precond_setup(dev(r), dev(q), d["blob_start"], s.a, 1.0, True)
    assert ei.value.name == "MB_ESINGULAR"
    assert "body 2" in str(ei.value)


def _solve_and_compare(ctx, s, prec, tol, u_tol, slip=None, wall=True):
    d = _dev_susp(s)
    U, W, lam, info = ctx.solve_mobility(
        d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"], s.a, s.eta, wall,
        None if slip is None else dev(slip), tol=tol, maxit=300, restart=100, prec=prec)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    Ur, Wr, lr = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, s.eta, wall, slip)
    assert info["converged"] == 1 and info["rel_residual"] <= tol
    assert rel_l2(host(U), Ur) <= u_tol, (rel_l2(host(U), Ur), info)
    assert rel_l2(host(W), Wr) <= u_tol, (rel_l2(host(W), Wr), info)
    assert rel_l2(host(lam), lr) <= 1e-5
    return info


def test_solve_fp64_small_suspension(ctx):
    """8 x 42-blob shells above the wall, FP64, tol 1e-10."""
    info = _solve_and_compare(ctx, I.config_small_suspension(1), "fp64", 1e-10, 1e-6)
    assert 3 <= info["iters"] <= 60


def test_solve_mixed_refinement_small_suspension(ctx):
    """FP32 pair kernel inside Arnoldi, FP64 restart residuals: same answer."""
    _solve_and_compare(ctx, I.config_small_suspension(1), "mixed", 1e-10, 1e-6)


def test_solve_df64_small_suspension(ctx):
    """Double-float pair kernel throughout: same answer as FP64."""
    _solve_and_compare(ctx, I.config_small_suspension(3), "df64", 1e-10, 1e-6)


def test_solve_mixed_monolayer_patch(ctx):
    """162-blob shells (global-memory factorisation path): mixed precision
    with double-float residuals reaches 1e-8; sampled residual rows checked
    with the oracle."""
    s = I.config_monolayer(2, n_bodies=24, box=14.0)
    d = _dev_susp(s)
    U, W, lam, info = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], d["F"],
                                         d["T"], s.a, 1.0, True, tol=1e-8, prec="mixed")
    assert info["converged"] == 1 and info["rel_residual"] <= 1e-8
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rows = np.random.default_rng(0).choice(s.n_blobs, 200, replace=False)
    res = O.residual_rows(rows, r, s.q, s.blob_start, host(lam), host(U), host(W), s.a)
    # ||b|| = ||(F, T)|| here (no slip); per-row residuals well below it
    bnorm = np.linalg.norm(np.concatenate([s.F, s.T]))
    assert np.abs(res).max() <= 1e-8 * bnorm
    Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, 1.0, True)
    assert rel_l2(host(U), Ur) <= 1e-6 and rel_l2(host(W), Wr) <= 1e-6


@pytest.mark.parametrize("restart", [60, 8])
def test_mixed_running_product_matches_fresh_residual(ctx, restart):
    """Mixed precision rebuilds A x from an FP64 running sum of M lambda whose
    small late increments come from the FP32 kernel.  The residual it reports
    must agree with a fresh FP64 product of the returned solution; restart = 8
    forces many short cycles and so many FP32 increments."""
    s = I.config_monolayer(3, n_bodies=16, box=12.0)
    d = _dev_susp(s)
    tol = 1e-8
    U, W, lam, info = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], d["F"],
                                         d["T"], s.a, 1.0, True, tol=tol, maxit=400,
                                         restart=restart, prec="mixed")
    assert info["converged"] == 1
    r = ctx.blob_positions(d["q"], d["theta"], d["blob_start"], d["rho"])
    Ml = ctx.mobility_matvec(r, lam, s.a, 1.0, True, "fp64")
    UO = torch.cat([U, W], 1).contiguous()
    rb = ctx.K_apply(r, d["q"], d["blob_start"], UO) - Ml
    rB = ctx.KT_apply(r, d["q"], d["blob_start"], lam) - torch.cat([d["F"], d["T"]], 1)
    bnorm = float(np.linalg.norm(np.concatenate([s.F, s.T])))
    fresh = float(torch.sqrt((rb * rb).sum() + (rB * rB).sum()).item()) / bnorm
    assert fresh <= 1.2 * tol
    assert abs(fresh - info["rel_residual"]) <= 0.2 * tol


def test_repeated_and_interleaved_solves_replay_captured_steps(ctx):
    """Small systems run each Arnoldi step as a CUDA graph from the second
    time the step is met on: three rounds of two interleaved problems in
    two precisions (record, capture, replay) agree with the first round to
    well within the solve tolerance (the double-float product's atomics
    make rounding differ from run to run)."""
    probs = [I.config_small_suspension(1), I.mixed_suspension(5, 10)]
    devs = [_dev_susp(s) for s in probs]
    first = {}
    for rnd in range(3):
        for k, (s, d) in enumerate(zip(probs, devs)):
            for prec in ("mixed", "fp64"):
                U, W, lam, info = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"],
                                                     d["F"], d["T"], s.a, s.eta, True, tol=1e-10,
                                                     prec=prec)
                assert info["converged"] == 1
                got = (host(U), host(W), host(lam))
                if rnd == 0:
                    first[(k, prec)] = got
                else:
                    for x, y in zip(got, first[(k, prec)]):
                        assert rel_l2(x, y) <= 1e-9


def test_wait_limit_returns_timeout_and_context_recovers(ctx):
    """With a host-wait limit far below a Krylov step (1 us), the solve
    returns MB_ETIMEOUT while its enqueued work still runs.  After a
    synchronisation and with the limit lifted, the same context solves the
    problem to the result it gave before.  A non-finite limit is refused."""
    s = I.config_small_suspension(1)
    d = _dev_susp(s)
    args = (d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"], s.a, s.eta, True)
    U0, W0, lam0, _ = ctx.solve_mobility(*args, tol=1e-10, prec="mixed")
    with pytest.raises(mb.MBError) as ei:
        ctx.set_wait_limit(float("nan"))
    assert ei.value.name == "MB_EINVAL"
    ctx.set_wait_limit(1e-6)
    try:
        with pytest.raises(mb.MBError) as ei:
            ctx.solve_mobility(*args, tol=1e-10, prec="mixed")
        assert ei.value.name == "MB_ETIMEOUT"
    finally:
        torch.cuda.synchronize()
        ctx.set_wait_limit(0.0)
    for _ in range(2):
        U, W, lam, info = ctx.solve_mobility(*args, tol=1e-10, prec="mixed")
        assert info["converged"] == 1
        for x, y in zip((U, W, lam), (U0, W0, lam0)):
            assert rel_l2(host(x), host(y)) <= 1e-9


def test_solve_fp32_small_suspension(ctx):
    _solve_and_compare(ctx, I.config_small_suspension(2), "fp32", 1e-6, 1e-5)


def test_solve_with_slip_and_free_space(ctx):
    s = I.config_small_suspension(4)
    slip = np.random.default_rng(5).standard_normal((s.n_blobs, 3)) * 0.1
    _solve_and_compare(ctx, s, "fp64", 1e-10, 1e-6, slip=slip)
    _solve_and_compare(ctx, s, "fp64", 1e-10, 1e-6, wall=False)


def test_solve_mixed_bodies(ctx):
    s = I.mixed_suspension(8, 16)
    _solve_and_compare(ctx, s, "mixed", 1e-10, 1e-6)


def test_solve_not_converged_reports_best_iterate(ctx):
    s = I.config_small_suspension(1)
    d = _dev_susp(s)
    U, W, lam, info = ctx.solve_mobility(
        d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"], s.a, s.eta, True,
        tol=1e-12, maxit=2, restart=100, prec="fp64", raise_on_nonconvergence=False)
    assert info["converged"] == 0 and info["iters"] == 2
    assert np.isfinite(host(U)).all() and info["rel_residual"] < 1.0
    with pytest.raises(mb.MBError) as ei:
        ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"], s.a,
                           s.eta, True, tol=1e-12, maxit=2, prec="fp64")
    assert ei.value.name == "MB_ENOTCONVERGED"


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_permeable_bodies_match_oracle(ctx, prec):
    """Appendix C: kappa_p / (eta dV_i) on the diagonal of M for every blob of
    a permeable body (one kappa per body, dV_i = 4 pi a^3 / 3); the GPU solve
    matches the oracle's direct solve of the shifted saddle system."""
    s = I.mixed_suspension(12, 8)
    kappa = np.random.default_rng(3).uniform(0.01, 2.0, s.n_bodies)
    per_blob = np.repeat(kappa, np.diff(s.blob_start))
    shift = per_blob / (4.0 * np.pi * s.a ** 3 / 3.0)
    d = _dev_susp(s)
    U, W, lam, info = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], d["F"],
                                         d["T"], s.a, 1.0, True, tol=1e-11, maxit=400,
                                         prec=prec, shift=dev(shift))
    assert info["converged"] == 1
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    Ur, Wr, lr = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, 1.0, True, shift=shift)
    assert rel_l2(host(U), Ur) <= 1e-8 and rel_l2(host(W), Wr) <= 1e-8
    assert rel_l2(host(lam), lr) <= 1e-7
    # zero permeability is the rigid body
    U0, _, _, _ = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], d["F"],
                                     d["T"], s.a, 1.0, True, tol=1e-11, maxit=400, prec="fp64",
                                     shift=dev(np.zeros(s.n_blobs)))
    Ur0, _, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, s.a, 1.0, True)
    assert rel_l2(host(U0), Ur0) <= 1e-8


def _shell_and_line():
    """A 42-blob shell (body 0) and three blobs on a line through the
    tracking point of body 1, which cannot resist spin about that line."""
    a = 0.243
    rho0 = I.shell(42)
    rho1 = np.array([[-2.2 * a, 0.0, 0.0], [0.0, 0.0, 0.0], [2.2 * a, 0.0, 0.0]])
    return I.Suspension(q=np.array([[0.0, 0.0, 3.0], [4.0, 0.0, 3.0]]),
                        theta=np.array([[1.0, 0, 0, 0], [1.0, 0, 0, 0]]),
                        blob_start=np.array([0, 42, 45], dtype=np.int64),
                        rho=np.concatenate([rho0, rho1]), F=np.array([[0.0, 0, -1], [0.1, 0, -1]]),
                        T=np.zeros((2, 3)), a=a)


def test_solve_reports_body_that_cannot_resist_a_rigid_motion(ctx):
    """K_p^T M_pp^-1 K_p is singular for blobs on a line through the tracking
    point (Section 2.1.2): the setup reports MB_ESINGULAR naming the body
    instead of solving with a meaningless inverse."""
    s = _shell_and_line()
    d = _dev_susp(s)
    with pytest.raises(mb.MBError) as ei:
        ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"], s.a,
                           1.0, True, tol=1e-10, prec="fp64")
    assert ei.value.name == "MB_ESINGULAR" and "body 1" in str(ei.value)
    # the resistance problem only needs M_pp^-1, which exists
    U = dev(np.array([[0.0, 0, 1.0], [0.0, 0, 1.0]]))
    F, T, lam, info = ctx.solve_resistance(d["q"], d["theta"], d["blob_start"], d["rho"], U,
                                           dev(np.zeros((2, 3))), s.a, 1.0, True, tol=1e-10)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    Fr, Tr, _ = O.solve_resistance(r, s.q, s.blob_start, host(U), np.zeros((2, 3)), s.a, 1.0, True)
    assert rel_l2(host(F), Fr) <= 1e-8


def test_zero_right_hand_side(ctx):
    """b = 0 is solved by x = 0 without iterations (mobility and resistance)."""
    s = I.config_small_suspension(2)
    d = _dev_susp(s)
    z = dev(np.zeros((s.n_bodies, 3)))
    for prec in ("fp64", "mixed"):
        U, W, lam, info = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], z, z,
                                             s.a, 1.0, True, tol=1e-10, prec=prec)
        assert info["converged"] == 1 and info["iters"] == 0
        assert np.all(host(U) == 0) and np.all(host(W) == 0) and np.all(host(lam) == 0)
        F, T, lam, info = ctx.solve_resistance(d["q"], d["theta"], d["blob_start"], d["rho"], z, z,
                                               s.a, 1.0, True, tol=1e-10, prec=prec)
        assert info["converged"] == 1 and np.all(host(F) == 0) and np.all(host(lam) == 0)
