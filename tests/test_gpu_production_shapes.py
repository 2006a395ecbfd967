"""Parity at the production shapes of the solver workloads.

- The sedimented monolayer's bodies (162-blob shells, a = 0.12, 486 rows per
  block) at its area density, with at least as many bodies as the GPU has
  SMs: the block-diagonal preconditioner of Section 2.2.2 is set up in
  several groups of bodies there, as it is for the 4,096-body workload, and
  kept in factored form (L, L^-1 K and the 6 x 6 Schur inverse), applied by
  triangular solves.
- Bodies of 64 blobs (192 rows), at least as many as SMs: the factorisation
  with one CTA per body and the rows in global memory, factored form.
- The whole 256-suspension batch (91,074 bodies, 2.6M blobs) in one
  mb_solve_batch call.

Bars: preconditioner applications within 1e-8 relative of the oracle's
per-body direct solve; solves to a true relative residual of 1e-8, checked on
sampled rows by the oracle (each row a full FP64 pass over all sources) and
on every body's force and torque balance; body velocities within 1e-6 of the
plain FP64 path and of the oracle's dense direct solve where it fits.
"""
import math

import numpy as np
import pytest
import torch

import paper_1602_02170_gb300 as mb
from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu


def _sm_count():
    return torch.cuda.get_device_properties(0).multi_processor_count


def _dev_susp(s):
    return dict(q=dev(s.q), theta=dev(s.theta), blob_start=dev(s.blob_start, torch.int64),
                rho=dev(s.rho), F=dev(s.F), T=dev(s.T))


def _monolayer_patch(seed=11):
    nb = max(_sm_count(), 160)
    # the monolayer's density: 4,096 bodies on a 200 x 200 patch
    return I.config_monolayer(seed, n_bodies=nb, box=200.0 * math.sqrt(nb / 4096.0))


def test_preconditioner_monolayer_shape_matches_oracle(ctx):
    s = _monolayer_patch()
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = np.random.default_rng(21)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, True)
    lam, UO = ctx.precond_apply(dev(w), dev(g))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, w, g)
    assert rel_l2(host(lam), lam_ref) <= 1e-8
    assert rel_l2(host(UO), UO_ref) <= 1e-8


def test_solve_monolayer_shape_mixed_matches_fp64_and_oracle_rows(ctx):
    s = _monolayer_patch(12)
    d = _dev_susp(s)
    args = (d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"], s.a, 1.0, True)
    U, W, lam, info = ctx.solve_mobility(*args, tol=1e-8, maxit=300, restart=60, prec="mixed")
    assert info["converged"] == 1 and info["rel_residual"] <= 1e-8
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    bnorm = np.linalg.norm(np.concatenate([s.F, s.T]))
    rows = np.random.default_rng(0).choice(s.n_blobs, 200, replace=False)
    res = O.residual_rows(rows, r, s.q, s.blob_start, host(lam), host(U), host(W), s.a)
    assert np.abs(res).max() <= 1e-8 * bnorm
    # force and torque balance of every body, -K^T lambda = -(F, T)
    Fo, To = O.KT_apply(host(lam), r, s.q, s.blob_start)
    assert np.abs(np.concatenate([Fo - s.F, To - s.T])).max() <= 1e-8 * bnorm
    U64, W64, _, info64 = ctx.solve_mobility(*args, tol=1e-8, maxit=300, restart=60, prec="fp64")
    assert info64["converged"] == 1
    assert rel_l2(host(U), host(U64)) <= 1e-6 and rel_l2(host(W), host(W64)) <= 1e-6


def _lattice_bodies(nbod, seed, shape=(4, 4, 4)):
    """nbod jittered cubic-lattice bodies of prod(shape) blobs (spacing 2.2 a,
    a = 0.1), spread along a line above the wall."""
    g = np.stack(np.meshgrid(*[np.arange(k) for k in shape], indexing="ij"), -1)
    a = 0.1
    rho1 = (g.reshape(-1, 3) - (np.array(shape) - 1) / 2.0) * (2.2 * a)
    rng = np.random.default_rng(seed)
    nbl = len(rho1)
    rho = np.concatenate([rho1 + 0.01 * a * rng.standard_normal(rho1.shape) for _ in range(nbod)])
    q = np.array([[2.5 * (k % 40), 2.5 * (k // 40), 1.2 + 0.1 * (k % 7)] for k in range(nbod)])
    return I.Suspension(q=q, theta=I.random_unit_quaternions(rng, nbod),
                        blob_start=np.arange(nbod + 1, dtype=np.int64) * nbl, rho=rho,
                        F=rng.normal(0.0, 0.1, (nbod, 3)) - [0.0, 0.0, 1.0],
                        T=rng.normal(0.0, 0.1, (nbod, 3)), a=a)


def test_preconditioner_many_mid_size_bodies_matches_oracle(ctx):
    """At least as many 64-blob bodies (192 rows) as SMs: one CTA per body,
    rows factored in global memory."""
    s = _lattice_bodies(max(_sm_count(), 160), 31)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    assert r[:, 2].min() > s.a
    rng = np.random.default_rng(32)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, True)
    lam, UO = ctx.precond_apply(dev(w), dev(g))
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, w, g)
    assert rel_l2(host(lam), lam_ref) <= 1e-8
    assert rel_l2(host(UO), UO_ref) <= 1e-8


def test_preconditioner_many_mid_size_bodies_singular_block_reported(ctx):
    """The same path reports an indefinite block (one blob at z = a/2) as
    MB_ESINGULAR naming the body."""
    s = _lattice_bodies(max(_sm_count(), 160), 33)
    k = 123
    q = s.q.copy()
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    q[k, 2] -= r[s.blob_start[k]:s.blob_start[k + 1], 2].min() - 0.5 * s.a
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    d = _dev_susp(s)
    with pytest.raises(mb.MBError) as ei:
        ctx.precond_setup(dev(r), dev(q), d["blob_start"], s.a, 1.0, True)
    assert ei.value.name == "MB_ESINGULAR"
    assert f"body {k}" in str(ei.value)


def test_solve_many_mid_size_bodies_matches_fp64(ctx):
    s = _lattice_bodies(max(_sm_count(), 160), 34)
    d = _dev_susp(s)
    args = (d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"], s.a, 1.0, True)
    U, W, lam, info = ctx.solve_mobility(*args, tol=1e-8, maxit=300, restart=60, prec="mixed")
    assert info["converged"] == 1
    U64, W64, _, _ = ctx.solve_mobility(*args, tol=1e-8, maxit=300, restart=60, prec="fp64")
    assert rel_l2(host(U), host(U64)) <= 1e-6 and rel_l2(host(W), host(W64)) <= 1e-6
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rows = np.random.default_rng(1).choice(s.n_blobs, 100, replace=False)
    res = O.residual_rows(rows, r, s.q, s.blob_start, host(lam), host(U), host(W), s.a)
    assert np.abs(res).max() <= 1e-8 * np.linalg.norm(np.concatenate([s.F, s.T]))


def test_full_batch_matches_solving_alone(ctx):
    """All 256 suspensions of the batched workload in one mb_solve_batch
    call (mixed precision, tol 1e-8): the four smallest and the two largest
    problems agree with solving each alone in FP64 (1e-6 relative), and the
    smallest with the oracle's dense direct solve."""
    susp = I.config_batched(1)
    probs = [_dev_susp(s) for s in susp]
    a = susp[0].a
    res = ctx.solve_batch(probs, a, tol=1e-8, maxit=300, restart=60, prec="mixed")
    assert all(r[3]["converged"] == 1 and r[3]["rel_residual"] <= 1e-8 for r in res)
    order = np.argsort([s.n_blobs for s in susp])
    picks = list(order[:4]) + list(order[-2:])
    for k in picks:
        P = probs[k]
        U, W, _, info = ctx.solve_mobility(P["q"], P["theta"], P["blob_start"], P["rho"], P["F"],
                                           P["T"], a, 1.0, True, tol=1e-8, maxit=300, restart=60,
                                           prec="fp64")
        assert rel_l2(host(res[k][0]), host(U)) <= 1e-6, (k, susp[k].n_blobs)
        assert rel_l2(host(res[k][1]), host(W)) <= 1e-6, (k, susp[k].n_blobs)
    s = susp[order[0]]
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, a, 1.0, True)
    assert rel_l2(host(res[order[0]][0]), Ur) <= 1e-6
    assert rel_l2(host(res[order[0]][1]), Wr) <= 1e-6


def test_resistance_inverts_mobility_on_factored_blocks(ctx):
    """At least as many 64-blob bodies as SMs (factored blocks, applied by
    triangular solves, with and without the body rows): the resistance
    problem (Eq. resistance_problem) given the velocities of a mobility
    solve returns the applied forces and torques."""
    s = _lattice_bodies(max(_sm_count(), 160), 35)
    d = _dev_susp(s)
    U, W, _, _ = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], d["F"], d["T"],
                                    s.a, 1.0, True, tol=1e-11, maxit=400, restart=100, prec="fp64")
    F, T, _, info = ctx.solve_resistance(d["q"], d["theta"], d["blob_start"], d["rho"], U, W, s.a,
                                         1.0, True, tol=1e-11, maxit=800, restart=200, prec="fp64")
    assert info["converged"] == 1
    assert rel_l2(host(F), s.F) <= 1e-8 and rel_l2(host(T), s.T) <= 1e-8


def test_preconditioner_four_bodies_per_sm_one_cta_path(ctx):
    """Four times as many 64-blob bodies as SMs: several one-CTA
    factorisations share each SM (the pivot of every column is read by all
    warps while one of them overwrites it with its square root; each warp
    must use the pivot itself).  The application matches the oracle."""
    s = _lattice_bodies(4 * _sm_count(), 36)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    rng = np.random.default_rng(37)
    w = rng.standard_normal((s.n_blobs, 3))
    g = rng.standard_normal((s.n_bodies, 6))
    d = _dev_susp(s)
    lam_ref, UO_ref = O.precond_apply(r, s.q, s.blob_start, s.a, 1.0, True, w, g)
    for _ in range(2):
        ctx.precond_setup(dev(r), d["q"], d["blob_start"], s.a, 1.0, True)
        lam, UO = ctx.precond_apply(dev(w), dev(g))
        assert rel_l2(host(lam), lam_ref) <= 1e-8
        assert rel_l2(host(UO), UO_ref) <= 1e-8
