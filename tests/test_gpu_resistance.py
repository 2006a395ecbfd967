"""Resistance problem (Eq. resistance_problem) on the GPU against the oracle's
dense direct solve, the effective-radius table and the mobility problem."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dev_susp(s):
    return dict(q=dev(s.q), theta=dev(s.theta), blob_start=dev(s.blob_start, torch.int64),
                rho=dev(s.rho))


def _motion(nb, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nb, 3)), rng.standard_normal((nb, 3)) * 0.5


@pytest.mark.parametrize("prec", ["fp64", "mixed", "df64"])
@pytest.mark.parametrize("precond", ["wall", "free_shared"])
def test_resistance_matches_oracle(ctx, prec, precond):
    for s in (I.config_small_suspension(3), I.mixed_suspension(4, 7)):
        d = _dev_susp(s)
        U, W = _motion(s.n_bodies, 1)
        slip = np.random.default_rng(2).standard_normal((s.n_blobs, 3)) * 0.1
        F, T, lam, info = ctx.solve_resistance(d["q"], d["theta"], d["blob_start"], d["rho"],
                                               dev(U), dev(W), s.a, 1.0, True, dev(slip),
                                               tol=1e-11, maxit=600, prec=prec, precond=precond)
        assert info["converged"] == 1
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        Fr, Tr, lr = O.solve_resistance(r, s.q, s.blob_start, U, W, s.a, 1.0, True, slip)
        assert rel_l2(host(F), Fr) <= 1e-8
        assert rel_l2(host(T), Tr) <= 1e-8
        assert rel_l2(host(lam), lr) <= 1e-7


def test_resistance_of_isotropic_shell_matches_table(ctx):
    """A 12-blob shell in an unbounded domain, translated and rotated: the GPU
    forces give R_h and R_tau of Table Stresslets_3D."""
    g = json.load(open(os.path.join(GOLDEN, "effective_radii.json")))
    for n, ratio, rh_ref, rt_ref in g["rows"]:
        if n != 12:
            continue
        rho = I.shell(12)
        a = ratio * I.min_spacing(rho)
        args = (dev(np.zeros((1, 3))), dev(np.array([[1.0, 0, 0, 0]])),
                dev(np.array([0, 12]), torch.int64), dev(rho))
        F, T, _, _ = ctx.solve_resistance(*args, dev([[0.0, 1.0, 0.0]]), dev(np.zeros((1, 3))), a,
                                          1.0, False, tol=1e-12)
        assert abs(host(F)[0, 1] / (6 * math.pi) - rh_ref) <= 1.5e-4
        F, T, _, _ = ctx.solve_resistance(*args, dev(np.zeros((1, 3))), dev([[0.0, 0.0, 1.0]]), a,
                                          1.0, False, tol=1e-12)
        assert abs((host(T)[0, 2] / (8 * math.pi)) ** (1 / 3) - rt_ref) <= 1.5e-4


def test_resistance_inverts_gpu_mobility(ctx):
    """Mobility then resistance on the GPU returns the applied forces."""
    s = I.mixed_suspension(9, 6)
    d = _dev_susp(s)
    U, W, lam, _ = ctx.solve_mobility(d["q"], d["theta"], d["blob_start"], d["rho"], dev(s.F),
                                      dev(s.T), s.a, 1.0, True, tol=1e-12, maxit=400, prec="fp64")
    F, T, lam2, _ = ctx.solve_resistance(d["q"], d["theta"], d["blob_start"], d["rho"], U, W, s.a,
                                         1.0, True, tol=1e-12, maxit=600, prec="fp64")
    assert rel_l2(host(F), s.F) <= 1e-8
    assert rel_l2(np.concatenate([host(F), host(T)]), np.concatenate([s.F, s.T])) <= 1e-8
    assert rel_l2(host(lam2), host(lam)) <= 1e-7


def test_public_apply_refuses_resistance_blocks(ctx):
    """After a resistance solve the context holds blob blocks only; the public
    indefinite apply reports that instead of returning wrong numbers."""
    s = I.config_small_suspension(1)
    d = _dev_susp(s)
    U, W = _motion(s.n_bodies, 3)
    ctx.solve_resistance(d["q"], d["theta"], d["blob_start"], d["rho"], dev(U), dev(W), s.a, 1.0,
                         True, tol=1e-8)
    import paper_1602_02170_gb300 as mb
    with pytest.raises(mb.MBError) as ei:
        ctx.precond_apply(dev(np.zeros((s.n_blobs, 3))), dev(np.zeros((s.n_bodies, 6))))
    assert ei.value.name == "MB_EINVAL"
