"""Parity of the pair kernel (u = M f, wall-corrected RPY) with the FP64 oracle.

Tolerances: FP64 path 1e-12 (rounding order only); FP32+Kahan path 1e-5
relative L2 and 1e-5 of max|u| element-wise — the matvec accuracy bar for the
FP32 path (FP32 pair arithmetic with hi/lo positions; expected ~1e-7);
double-float path 1e-10 (about 46 significant bits per operation, positions
carried as hi + lo FP32 pairs, i.e. to ~2^-48 of their magnitude).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_1602_02170_gb300 import inputs as I
from tests.gpu_common import ctx, dev, host, rel_l2  # noqa: F401

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "df64": 1e-10}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df64"])
@pytest.mark.parametrize("wall", [True, False])
@pytest.mark.parametrize("n", [1, 7, 255, 256, 1537, 5000, 9000])
def test_matvec_small_elementwise(ctx, prec, wall, n):
    """Sizes spanning one partial tile, exact tiles and several tiles plus a
    ragged tail, against the oracle element by element."""
    r, f = I.blob_cloud(100 + n, n, 0.5, 3.0 * max(1.0, n ** 0.5 / 3), 0.5, 1.5)
    ref = O.matvec(r, f, 0.5, 1.0, wall)
    got = host(ctx.mobility_matvec(dev(r), dev(f), 0.5, 1.0, wall, prec))
    tol = TOL[prec]
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()
    assert rel_l2(got, ref) <= tol


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df64"])
def test_matvec_overlaps_coincident_and_contact(ctx, prec):
    """Degenerate pairs: coincident distinct blobs (r = 0), exact contact
    r = 2a, deep overlaps, and blobs at z = a touching the wall."""
    a = 0.5
    r = np.array(
        [[1.0, 1.0, 0.7], [1.0, 1.0, 0.7], [2.0, 1.0, 0.7], [3.0, 1.0, 0.7], [3.1, 1.05, 0.75],
         [5.0, 5.0, a], [5.0, 5.0 + 2 * a, a], [7.0, 2.0, 2.5]]
    )
    f = np.random.default_rng(0).standard_normal(r.shape)
    for wall in (True, False):
        ref = O.matvec(r, f, a, 1.0, wall)
        got = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, wall, prec))
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()


@pytest.fixture(scope="module")
def full_size_case():
    """The 65,536-blob workload and the oracle on 4,096 sampled targets."""
    r, f, a = I.config_matvec_cloud(1)
    rows = np.random.default_rng(7).choice(r.shape[0], 4096, replace=False)
    return r, f, a, rows, O.matvec(r, f, a, 1.0, True, targets=rows)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "df64"])
def test_matvec_full_size_sampled(ctx, full_size_case, prec):
    """The 65,536-blob workload (a = 0.5, xy in [0,400]^2, z in [a,3a]) in
    the launch configuration the benchmark times, checked on 4,096 sampled
    targets against the oracle over all sources."""
    r, f, a, rows, ref = full_size_case
    got = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, prec))
    assert rel_l2(got[rows], ref) <= TOL[prec]
    assert np.abs(got[rows] - ref).max() <= TOL[prec] * np.abs(ref).max()


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("n", [7, 513, 1537, 4100, 9000])
def test_matvec_fp32_variants_elementwise(ctx, variant, n):
    """Every FP32 kernel variant (scalar; packed with 2 or 4 targets per
    thread; symmetric over block pairs) against the oracle, on sizes that
    leave ragged blocks (513 = one full block pair plus a single blob)."""
    r, f = I.blob_cloud(300 + n, n, 0.5, 3.0 * max(1.0, n ** 0.5 / 3), 0.5, 1.5)
    ref = O.matvec(r, f, 0.5, 1.0, True)
    ctx.set_pair_variant(variant)
    try:
        got = host(ctx.mobility_matvec(dev(r), dev(f), 0.5, 1.0, True, "fp32"))
    finally:
        ctx.set_pair_variant(-1)
    assert np.abs(got - ref).max() <= TOL["fp32"] * np.abs(ref).max()
    assert rel_l2(got, ref) <= TOL["fp32"]


def test_autotuner_picks_a_variant_and_keeps_it(ctx):
    r, f, a = I.config_matvec_cloud(5, n=20000)
    assert ctx.pair_variant(20000, True) in (-1, 0, 1, 2)
    u1 = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, "fp32"))
    v = ctx.pair_variant(20000, True)
    assert v in (0, 1, 2, 3, 4)
    u2 = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, "fp32"))
    # the symmetric variant adds partial sums with FP64 atomics: equal to FP64 rounding
    np.testing.assert_allclose(u1, u2, rtol=1e-13, atol=1e-15 * np.abs(u1).max())
    assert ctx.pair_variant(20000, True) == v


def test_symmetric_variant_full_size_sampled(ctx, full_size_case):
    """The symmetric kernel on the 65,536-blob workload against the oracle."""
    r, f, a, rows, ref = full_size_case
    ctx.set_pair_variant(3)
    try:
        got = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, "fp32"))
    finally:
        ctx.set_pair_variant(-1)
    assert rel_l2(got[rows], ref) <= TOL["fp32"]
    assert np.abs(got[rows] - ref).max() <= TOL["fp32"] * np.abs(ref).max()


def test_matvec_translation_parallel_to_wall(ctx):
    """Property at any size: shifting every blob parallel to the wall by
    (+300, -200) leaves u unchanged (FP32 path keeps it thanks to hi/lo)."""
    r, f, a = I.config_matvec_cloud(2, n=20000)
    u0 = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, "fp32"))
    r2 = r + np.array([300.0, -200.0, 0.0])
    u1 = host(ctx.mobility_matvec(dev(r2), dev(f), a, 1.0, True, "fp32"))
    assert rel_l2(u1, u0) <= 1e-6


def test_matvec_host_pointers_match_device(ctx):
    """Host-pointer calls stage through the library and give the same bits."""
    r, f = I.blob_cloud(3, 3000, 0.5, 40.0, 0.5, 1.5)
    ud = host(ctx.mobility_matvec(dev(r), dev(f), 0.5, 1.0, True, "fp32"))
    rh = torch.from_numpy(r).pin_memory()
    fh = torch.from_numpy(f).pin_memory()
    uh = ctx.mobility_matvec(rh, fh, 0.5, 1.0, True, "fp32").numpy()
    np.testing.assert_allclose(uh, ud, rtol=1e-13, atol=1e-15 * np.abs(ud).max())


def test_matvec_empty_and_errors(ctx):
    import paper_1602_02170_gb300 as mb

    e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    out = ctx.mobility_matvec(e, e, 0.5)
    assert out.shape == (0, 3)
    r = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(mb.MBError) as ei:
        ctx.mobility_matvec(r, r, -1.0)
    assert ei.value.name == "MB_EINVAL"
    with pytest.raises(mb.MBError):
        ctx.mobility_matvec(r, r.cpu(), 0.5)


@pytest.mark.parametrize("layout", ["monolayer", "line"])
def test_symmetric_variant_spatial_order(ctx, layout):
    """From 16,384 blobs the symmetric kernels run in a spatial order (cells
    of a grid in Morton order).  In FP32 block pairs far apart skip the lo
    parts of the separations and the overlap test; in double-float, block
    pairs 64 a apart sum the t4 terms of the wall polynomials in FP32.
    Bodies of the monolayer (clustered blobs, many overlapping pairs within a
    shell) and blobs spread along one line (one axis takes every bit of the
    grid) both match the FP64 kernel over all rows and the oracle on sampled
    rows, each precision at its own bound."""
    if layout == "monolayer":
        s = I.config_monolayer(13, n_bodies=120, box=200.0 * (120 / 4096.0) ** 0.5)
        r = O.blob_positions(s.q, s.theta, s.blob_start, s.rho)
        a = s.a
    else:
        n = 18000
        rng = np.random.default_rng(14)
        r = np.stack([np.sort(rng.uniform(-500.0, 900.0, n)), rng.uniform(-1.0, 1.0, n),
                      rng.uniform(0.6, 1.5, n)], axis=1)
        a = 0.5
    f = np.random.default_rng(15).standard_normal(r.shape)
    assert r.shape[0] >= 16384
    ctx.set_pair_variant(3)
    try:
        got = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, "fp32"))
    finally:
        ctx.set_pair_variant(-1)
    ref64 = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, "fp64"))
    assert rel_l2(got, ref64) <= TOL["fp32"]
    rows = np.random.default_rng(16).choice(r.shape[0], 1500, replace=False)
    ref = O.matvec(r, f, a, 1.0, True, targets=rows)
    assert rel_l2(got[rows], ref) <= TOL["fp32"]
    assert np.abs(got[rows] - ref).max() <= TOL["fp32"] * np.abs(ref).max()
    # the double-float kernel in the same order: block pairs 64 a apart sum
    # their t4 terms in FP32; the agreement stays at double-float rounding
    got_df = host(ctx.mobility_matvec(dev(r), dev(f), a, 1.0, True, "df64"))
    assert rel_l2(got_df, ref64) <= 1e-12
    assert rel_l2(got_df[rows], ref) <= 1e-12
