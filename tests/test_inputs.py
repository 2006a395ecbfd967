"""The seeded generators produce the workloads' stated geometry."""
import numpy as np
import pytest

from paper_1602_02170_gb300 import inputs as I


@pytest.mark.parametrize("n", [12, 42, 162, 642])
def test_shell_counts_and_radius(n):
    rho = I.shell(n, radius=1.5)
    assert rho.shape == (n, 3)
    np.testing.assert_allclose(np.linalg.norm(rho, axis=1), 1.5, rtol=1e-14)
    assert abs(rho.mean(axis=0)).max() < 1e-12


def test_shell_spacings():
    """Minimal spacing of the unit shells (used to set a = s/2 or s/4)."""
    for n, s in [(12, 1.05146), (42, 0.54653), (162, 0.27590)]:
        assert abs(I.min_spacing(I.shell(n)) - s) < 1e-5


def test_boomerang_geometry():
    rho = I.boomerang15()
    assert rho.shape == (15, 3)
    assert abs(rho.mean(axis=0)).max() < 1e-14
    assert abs(I.min_spacing(rho) - 0.3) < 1e-12
    corner = rho[0]
    assert abs(np.linalg.norm(rho[7] - corner) - 2.1) < 1e-12
    assert abs(np.linalg.norm(rho[14] - corner) - 2.1) < 1e-12
    assert abs(np.dot(rho[7] - corner, rho[14] - corner)) < 1e-12


def test_quaternions_unit_and_seeded():
    q1 = I.random_unit_quaternions(np.random.default_rng(3), 50)
    q2 = I.random_unit_quaternions(np.random.default_rng(3), 50)
    np.testing.assert_array_equal(q1, q2)
    np.testing.assert_allclose(np.linalg.norm(q1, axis=1), 1.0, rtol=1e-15)


def test_small_suspension_layout():
    s = I.config_small_suspension(1)
    assert s.n_bodies == 8 and s.n_blobs == 336
    assert s.blob_start.dtype == np.int64 and s.blob_start[-1] == 336
    assert (s.q[:, :2] >= 0).all() and (s.q[:, :2] <= 10).all()
    assert (s.q[:, 2] >= 1.5).all() and (s.q[:, 2] <= 4).all()
    d = np.linalg.norm(s.q[:, None] - s.q[None], axis=-1) + np.eye(8) * 99
    assert d.min() >= 2 * (1 + s.a)


def test_matvec_cloud():
    r, f, a = I.config_matvec_cloud(1, n=4096)
    assert r.shape == (4096, 3) and a == 0.5
    assert r[:, 2].min() >= a and r[:, 2].max() <= 3 * a


def test_mixed_suspension_blobs_above_wall():
    from scipy.spatial.transform import Rotation

    s = I.mixed_suspension(5, 20)
    for p in range(s.n_bodies):
        lo, hi = s.blob_start[p], s.blob_start[p + 1]
        th = s.theta[p]
        R = Rotation.from_quat([th[1], th[2], th[3], th[0]]).as_matrix()
        z = s.q[p, 2] + (s.rho[lo:hi] @ R.T)[:, 2]
        assert z.min() >= s.a - 1e-12


def test_monolayer_layout():
    """Sedimented monolayer: 4,096 shells of 162 blobs (N = 663,552, a = 0.12),
    centres in the 200 x 200 patch at heights [1.2, 1.6] without overlap,
    gravity forces and N(0, 0.1^2) torques."""
    from scipy.spatial import cKDTree

    s = I.config_monolayer(1)
    assert s.n_bodies == 4096 and s.n_blobs == 663552 and s.a == 0.12
    assert (np.diff(s.blob_start) == 162).all()
    assert (s.q[:, :2] >= 0).all() and (s.q[:, :2] <= 200).all()
    assert (s.q[:, 2] >= 1.2).all() and (s.q[:, 2] <= 1.6).all()
    assert (s.q[:, 2] - 1.0 >= s.a).all()  # the lowest blob of a unit shell stays above z = a
    d, _ = cKDTree(s.q).query(s.q, k=2)
    assert d[:, 1].min() >= 2 * (1 + s.a) - 1e-12
    np.testing.assert_array_equal(s.F, np.tile([0.0, 0.0, -1.0], (4096, 1)))
    assert abs(s.T.std() - 0.1) < 0.005 and abs(s.T.mean()) < 0.005


def test_batched_suspensions():
    """Batched workload: mixed suspensions (42-blob shells and 15-blob
    boomerangs) whose body counts are log-uniform in [8, 2048]."""
    batch = I.config_batched(1, n_problems=24)
    nb = np.array([s.n_bodies for s in batch])
    assert nb.min() >= 8 and nb.max() <= 2048
    logs = np.log(nb)
    assert np.log(8) <= logs.mean() <= np.log(2048)
    for s in batch:
        sizes = np.diff(s.blob_start)
        assert set(np.unique(sizes)) <= {15, 42}
        assert s.blob_start[-1] == s.n_blobs and s.a == 0.1625
        assert (s.q[:, 2] >= 1.2).all() and (s.q[:, 2] <= 3.0).all()
    assert nb.min() < 64 and nb.max() > 512  # the draw spans the range


def test_serving_requests_span_the_blob_range():
    """Serving requests: blob counts log-uniform in [100, 200,000] (bodies of
    28.5 blobs on average), each a valid mixed suspension."""
    reqs = [I.config_serving_request(s) for s in range(12)]
    sizes = np.array([r.n_blobs for r in reqs])
    assert sizes.min() >= 15 and sizes.max() <= 200_000 * 1.1
    assert sizes.min() < 1_000 and sizes.max() > 50_000
    for r in reqs:
        assert r.blob_start[-1] == r.n_blobs
        assert set(np.unique(np.diff(r.blob_start))) <= {15, 42}
