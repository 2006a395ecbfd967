"""Flow evaluation at points other than the blobs (targets != sources) and
the flow rendering of Appendix B, on the GPU against the oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("wall", [True, False])
@pytest.mark.parametrize("nt,ns", [(1, 1), (7, 1000), (1537, 513), (3000, 9000)])
def test_eval_matches_oracle(ctx, prec, wall, nt, ns):
    rng = np.random.default_rng(nt + ns)
    a = 0.4
    r, f = I.blob_cloud(int(ns), ns, a, 30.0, a, 3 * a)
    x = np.column_stack([rng.uniform(-2, 32, nt), rng.uniform(-2, 32, nt),
                         rng.uniform(0.2 * a, 5 * a, nt)])
    u = ctx.mobility_eval(dev(x), dev(r), dev(f), a, 1.0, wall, prec)
    ref = O.eval_points(x, r, f, a, 1.0, wall)
    if prec == "fp64":
        assert rel_l2(host(u), ref) <= TOL[prec]
    else:
        # FP32 rounding is relative to the terms, not to their sum: near the
        # wall a far source's Stokeslet and image nearly cancel (a single far
        # pair can lose two digits), so the scale is the unbounded-domain flow
        free = O.eval_points(x, r, f, a, 1.0, False)
        assert np.linalg.norm(host(u) - ref) <= TOL[prec] * np.linalg.norm(free)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_eval_at_blobs_is_the_matvec(ctx, prec):
    r, f = I.blob_cloud(3, 2500, 0.5, 40.0, 0.5, 1.5)
    u = ctx.mobility_eval(dev(r), dev(r), dev(f), 0.5, 1.0, True, prec)
    m = ctx.mobility_matvec(dev(r), dev(f), 0.5, 1.0, True, prec)
    assert rel_l2(host(u), host(m)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_render_flow_matches_oracle(ctx, prec):
    s = I.config_small_suspension(2)
    r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
    lam = np.random.default_rng(5).standard_normal((s.n_blobs, 3))
    off = I.shell(12) * s.a
    rng = np.random.default_rng(6)
    x = np.column_stack([rng.uniform(-1, 11, 800), rng.uniform(-1, 11, 800), rng.uniform(0.3, 5, 800)])
    v = ctx.render_flow(dev(x), dev(r), dev(lam), dev(off), 0.25 * s.a, 1.0, True, prec)
    ref = O.render_flow(x, r, lam, off, 0.25 * s.a, 1.0, True)
    assert rel_l2(host(v), ref) <= TOL[prec]


def test_eval_rejects_host_pointers_and_handles_no_blobs(ctx):
    import paper_1602_02170_gb300 as mb
    r = np.zeros((4, 3))
    r[:, 2] = 1.0
    p = r.ctypes.data
    st = ctx.L.mb_mobility_eval(ctx.handle, p, 4, p, p, 4, 0.5, 1.0, 1, 1, p, None)
    assert mb.STATUS[st] == "MB_EINVAL"
    u = ctx.mobility_eval(dev(np.ones((5, 3))), dev(np.zeros((0, 3))), dev(np.zeros((0, 3))), 0.5)
    assert np.all(host(u) == 0.0)
