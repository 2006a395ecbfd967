"""Active slip on the GPU (the slip right-hand side of Eq. saddle_M): a
squirmer's swimming speed (Section 4.3) and the stresslet radius under an
applied strain slip (Section 4.1, Table Stresslets_3D), against the oracle
and the paper's table."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401
from tests.test_oracle_pins import _strain_slip, squirmer_slip

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _one_body(rho):
    n = len(rho)
    return (dev(np.zeros((1, 3))), dev(np.array([[1.0, 0.0, 0.0, 0.0]])),
            dev(np.array([0, n]), torch.int64), dev(rho))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_squirmer_speed_matches_oracle_and_converges(ctx, prec):
    speeds = []
    for n in (162, 642):
        rho = I.shell(n)
        a = 0.5 * I.min_spacing(rho)
        q, th, bs, rh = _one_body(rho)
        z = dev(np.zeros((1, 3)))
        U, W, lam, info = ctx.solve_mobility(q, th, bs, rh, z, z, a, 1.0, False,
                                             dev(squirmer_slip(rho)), tol=1e-11, maxit=400,
                                             prec=prec)
        zz = np.zeros((1, 3))
        Ur, Wr, _ = O.solve_saddle(rho, zz, np.array([0, n]), zz, zz, a, 1.0, False,
                                   squirmer_slip(rho))
        assert abs(host(U)[0, 2] - Ur[0, 2]) <= 1e-8 * abs(Ur[0, 2])
        assert np.abs(host(U)[0, :2]).max() <= 1e-8 and np.abs(host(W)).max() <= 1e-8
        speeds.append((host(U)[0, 2] / (2.0 / 3.0) - 1.0, a))
    (e1, a1), (e2, a2) = speeds
    assert 0 < e2 < e1 and abs((e2 / a2) / (e1 / a1) - 1.0) <= 0.05


def test_stresslet_radii_match_table(ctx):
    g = json.load(open(os.path.join(GOLDEN, "stresslet_radii.json")))
    for n, ratio, rs_ref in g["rows"]:
        rho = I.shell(int(n))
        a = ratio * I.min_spacing(rho)
        q, th, bs, rh = _one_body(rho)
        z = dev(np.zeros((1, 3)))
        U, W, lam, _ = ctx.solve_mobility(q, th, bs, rh, z, z, a, 1.0, False,
                                          dev(_strain_slip(rho)), tol=1e-12, maxit=400,
                                          prec="fp64")
        S = host(ctx.lambda_moments(rh, q, bs, lam))[0]
        s = 0.5 * (S + S.T) - np.trace(S) / 3.0 * np.eye(3)
        rs = (-3.0 * s[0, 0] / (20.0 * math.pi)) ** (1.0 / 3.0)
        assert abs(rs - rs_ref) <= 1.5e-4, (n, ratio, rs, rs_ref)


def test_lambda_moments_match_definition(ctx):
    """S_p = sum_i lambda_i (x) (r_i - q_p) for a multi-body suspension."""
    s = I.mixed_suspension(3, 6)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    lam = np.random.default_rng(1).standard_normal((s.n_blobs, 3))
    S = host(ctx.lambda_moments(dev(r), dev(s.q), dev(s.blob_start, torch.int64), dev(lam)))
    for p in range(s.n_bodies):
        lo, hi = s.blob_start[p], s.blob_start[p + 1]
        ref = lam[lo:hi].T @ (r[lo:hi] - s.q[p])
        np.testing.assert_allclose(S[p], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    # the antisymmetric part is the torque K^T gives
    T = np.stack([S[:, 2, 1] - S[:, 1, 2], S[:, 0, 2] - S[:, 2, 0], S[:, 1, 0] - S[:, 0, 1]], 1)
    _, Tref = O.KT_apply(lam, r, s.q, s.blob_start)
    np.testing.assert_allclose(T, Tref, rtol=1e-10, atol=1e-10)
