"""Batched solves (mb_solve_batch) against individual solves and the oracle.

Bars: body velocities within 1e-6 relative of the oracle's direct solve and
of the same problem solved alone; a problem's result must not depend on the
other problems in its batch.
"""
import numpy as np
import pytest
import torch

import paper_1602_02170_gb300 as mb
from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu
A = 0.1625  # one blob radius for the mixed sphere/boomerang suspensions


def _prob(s, slip=None):
    d = dict(q=dev(s.q), theta=dev(s.theta), blob_start=dev(s.blob_start, torch.int64),
             rho=dev(s.rho), F=dev(s.F), T=dev(s.T))
    if slip is not None:
        d["slip"] = dev(slip)
    return d


def _suspensions():
    out = [I.mixed_suspension(40 + k, nb) for k, nb in enumerate([1, 3, 5, 8, 13, 21])]
    out.append(I.sphere_suspension(9, 8, 42, A, 10.0, 1.5, 4.0))
    return out


def test_batch_matches_alone_and_oracle(ctx):
    susp = _suspensions()
    res = ctx.solve_batch([_prob(s) for s in susp], A, 1.0, True, tol=1e-10, prec="mixed")
    for k, (s, (U, W, lam, info)) in enumerate(zip(susp, res)):
        assert info["converged"] == 1 and info["rel_residual"] <= 1e-10, (k, info)
        p = _prob(s)
        Ua, Wa, la, _ = ctx.solve_mobility(p["q"], p["theta"], p["blob_start"], p["rho"], p["F"],
                                           p["T"], A, 1.0, True, tol=1e-10, prec="mixed")
        assert rel_l2(host(U), host(Ua)) <= 1e-6, k
        assert rel_l2(host(W), host(Wa)) <= 1e-6, k
        if s.n_blobs <= 400:
            r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
            Ur, Wr, lr = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True)
            assert rel_l2(host(U), Ur) <= 1e-6, k
            assert rel_l2(host(W), Wr) <= 1e-6, k
            assert rel_l2(host(lam), lr) <= 1e-5, k


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_batch_each_tile_shape(ctx, variant):
    """The engine's FP32 tile shapes (packed with 2 or 4 targets per thread,
    symmetric over block pairs) give the same answer; problems of 20-40
    bodies span several 512-blob blocks."""
    susp = [I.mixed_suspension(600 + k, nb) for k, nb in enumerate([20, 33, 7, 40])]
    ctx.set_pair_variant(variant)
    try:
        res = ctx.solve_batch([_prob(s) for s in susp], A, tol=1e-10, prec="mixed")
    finally:
        ctx.set_pair_variant(-1)
    for s, (U, W, lam, info) in zip(susp, res):
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True)
        assert info["converged"] == 1
        assert rel_l2(host(U), Ur) <= 1e-6 and rel_l2(host(W), Wr) <= 1e-6


def test_batch_result_independent_of_companions(ctx):
    """The same problem solved in two different batches gives the same answer."""
    susp = _suspensions()
    target = susp[4]
    r1 = ctx.solve_batch([_prob(s) for s in susp], A, tol=1e-10, prec="mixed")[4]
    r2 = ctx.solve_batch([_prob(target), _prob(susp[0])], A, tol=1e-10, prec="mixed")[0]
    assert rel_l2(host(r1[0]), host(r2[0])) <= 1e-7
    assert rel_l2(host(r1[1]), host(r2[1])) <= 1e-7


@pytest.mark.parametrize("prec,tol,bar", [("fp64", 1e-10, 1e-6), ("fp32", 1e-6, 1e-5)])
def test_batch_precisions(ctx, prec, tol, bar):
    susp = _suspensions()[2:5]
    res = ctx.solve_batch([_prob(s) for s in susp], A, tol=tol, prec=prec)
    for s, (U, W, lam, info) in zip(susp, res):
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True)
        assert info["converged"] == 1
        assert rel_l2(host(U), Ur) <= bar and rel_l2(host(W), Wr) <= bar


def test_batch_with_slip(ctx):
    s = I.mixed_suspension(77, 6)
    slip = 0.1 * np.random.default_rng(1).standard_normal((s.n_blobs, 3))
    (U, W, lam, info), = ctx.solve_batch([_prob(s, slip)], A, tol=1e-10, prec="fp64")
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    Ur, Wr, _ = O.solve_saddle(r, s.q, s.blob_start, s.F, s.T, A, 1.0, True, slip)
    assert rel_l2(host(U), Ur) <= 1e-6 and rel_l2(host(W), Wr) <= 1e-6


def test_batch_reports_malformed_and_singular(ctx):
    susp = _suspensions()[1:4]
    probs = [_prob(s) for s in susp]
    bad = dict(probs[1])
    bs = susp[1].blob_start.copy()
    bs[-1] -= 1
    bad["blob_start"] = dev(bs, torch.int64)
    with pytest.raises(mb.MBError) as ei:
        ctx.solve_batch([probs[0], bad, probs[2]], A)
    assert ei.value.name == "MB_EINVAL" and "problem 1" in str(ei.value)
    # a body pushed down so that a blob sits at z = a/2: not positive definite
    s = susp[2]
    q = s.q.copy()
    r = O.blob_positions(q, s.theta, s.blob_start, s.rho)
    lo, hi = s.blob_start[0], s.blob_start[1]
    q[0, 2] -= r[lo:hi, 2].min() - 0.5 * A
    sing = dict(_prob(s))
    sing["q"] = dev(q)
    with pytest.raises(mb.MBError) as ei:
        ctx.solve_batch([probs[0], probs[1], sing], A)
    assert ei.value.name == "MB_ESINGULAR" and "problem 2" in str(ei.value)


def test_batch_not_converged(ctx):
    susp = _suspensions()[3:6]
    res = ctx.solve_batch([_prob(s) for s in susp], A, tol=1e-12, maxit=2, prec="fp64",
                          raise_on_nonconvergence=False)
    for U, W, lam, info in res:
        assert info["converged"] == 0 and info["iters"] == 2
        assert np.isfinite(host(U)).all()


def test_batch_with_a_zero_force_problem(ctx):
    """A problem with b = 0 finishes at admission with zeros; its companions
    are unaffected."""
    s0 = I.config_small_suspension(1)
    s1 = I.config_small_suspension(2)
    P0 = _prob(s0)
    P1 = _prob(s1)
    P1["F"] = torch.zeros_like(P1["F"])
    P1["T"] = torch.zeros_like(P1["T"])
    res = ctx.solve_batch([P0, P1], s0.a, tol=1e-10, prec="mixed")
    U1, W1, lam1, info1 = res[1]
    assert info1["converged"] == 1 and info1["iters"] == 0
    assert torch.count_nonzero(U1) == 0 and torch.count_nonzero(lam1) == 0
    alone = ctx.solve_batch([P0], s0.a, tol=1e-10, prec="mixed")[0]
    assert rel_l2(host(res[0][0]), host(alone[0])) <= 1e-9
