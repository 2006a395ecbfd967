"""Seeded synthetic inputs for the rigid multiblob mobility problem.

This module is the one piece shared by the CUDA path and the FP64 oracle.
It holds geometry and random draws only — reference blob offsets of each body
shape, body centres and orientations, forces and torques — and none of the
method's arithmetic: it never builds blob positions from (q, theta), never
evaluates a mobility, and never applies K or K^T.  Both sides receive the same
arrays and compute everything else themselves.

Body shapes (reference configuration, tracking point at the origin):
  * icosahedral shells: 12 blobs at the vertices of an icosahedron, refined by
    placing a blob at every edge midpoint and projecting it onto the sphere,
    giving 10*4**k + 2 blobs after k refinements (Section 4, "Results:
    Unbounded Domain", shell construction);
  * the 15-blob boomerang: two 8-blob arms at a right angle that share the
    corner blob (Section 6.4); arm length 2.1, spacing 0.3, tracking point at
    the blob centroid.

All random draws use numpy's PCG64 generator seeded by the caller.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "icosahedral_shell",
    "shell",
    "min_spacing",
    "boomerang15",
    "random_unit_quaternions",
    "Suspension",
    "blob_cloud",
    "sphere_suspension",
    "mixed_suspension",
    "config_small_suspension",
    "config_matvec_cloud",
    "config_monolayer",
    "config_batched",
    "config_serving_request",
]


# --------------------------------------------------------------------------
# body shapes
# --------------------------------------------------------------------------
def _icosahedron():
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
            [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
            [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
        ],
        dtype=np.float64,
    )
    f = [
        (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
        (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
        (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
        (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
    ]
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosahedral_shell(levels: int, radius: float = 1.0) -> np.ndarray:
    """Blob offsets of an icosahedral shell refined `levels` times.

    Returns an array of shape (10*4**levels + 2, 3) of points on the sphere of
    the given geometric radius R_g, centred at the origin.
    """
    if levels < 0:
        raise ValueError("levels must be >= 0")
    verts, faces = _icosahedron()
    verts = [tuple(x) for x in verts]
    for _ in range(levels):
        cache: dict = {}
        new_faces = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = (np.asarray(verts[i]) + np.asarray(verts[j])) * 0.5
                m /= np.linalg.norm(m)
                verts.append(tuple(m))
                cache[key] = len(verts) - 1
            return cache[key]

        for (i, j, k) in faces:
            a, b, c = mid(i, j), mid(j, k), mid(k, i)
            new_faces += [(i, a, c), (j, b, a), (k, c, b), (a, b, c)]
        faces = new_faces
    out = np.asarray(verts, dtype=np.float64) * radius
    assert out.shape[0] == 10 * 4**levels + 2
    return out


_SHELL_LEVEL = {12: 0, 42: 1, 162: 2, 642: 3, 2562: 4}


def shell(n_blobs: int, radius: float = 1.0) -> np.ndarray:
    """Icosahedral shell with 12, 42, 162, 642 or 2562 blobs."""
    if n_blobs not in _SHELL_LEVEL:
        raise ValueError(f"no icosahedral shell with {n_blobs} blobs")
    return icosahedral_shell(_SHELL_LEVEL[n_blobs], radius)


def min_spacing(rho: np.ndarray) -> float:
    """Smallest distance between two distinct blobs of one body."""
    d = np.linalg.norm(rho[:, None, :] - rho[None, :, :], axis=-1)
    d[np.diag_indices_from(d)] = np.inf
    return float(d.min())


def boomerang15(arm_length: float = 2.1) -> np.ndarray:
    """15-blob boomerang: two 8-blob arms at 90 degrees sharing the corner.

    The corner blob is the first; arm one runs along +x and arm two along +y
    in the reference frame.  Offsets are relative to the blob centroid, the
    tracking point used for this body.
    """
    s = arm_length / 7.0
    pts = [(0.0, 0.0, 0.0)]
    pts += [(s * k, 0.0, 0.0) for k in range(1, 8)]
    pts += [(0.0, s * k, 0.0) for k in range(1, 8)]
    pts = np.asarray(pts, dtype=np.float64)
    return pts - pts.mean(axis=0)


# --------------------------------------------------------------------------
# random draws
# --------------------------------------------------------------------------
def random_unit_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions, scalar first (s, x, y, z)."""
    g = rng.standard_normal((n, 4))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g


def _lowest_blob_height(theta: np.ndarray, rho: np.ndarray) -> float:
    """Lowest body-frame z offset after the rotation `theta`.

    Used only to reject orientations that would put a blob below the wall.
    The rotation is delegated to scipy (a library routine, scalar-last
    convention) so that this module carries none of the method's arithmetic.
    """
    from scipy.spatial.transform import Rotation

    rot = Rotation.from_quat([theta[1], theta[2], theta[3], theta[0]])
    return float(rot.apply(rho)[:, 2].min())


@dataclasses.dataclass
class Suspension:
    """A configuration of rigid multiblob bodies above a no-slip wall at z=0.

    q          (n_b, 3)   tracking points
    theta      (n_b, 4)   unit quaternions, scalar first
    blob_start (n_b + 1,) int64 CSR offsets: body p owns blobs
                          blob_start[p] .. blob_start[p+1]-1
    rho        (N, 3)     reference-frame blob offsets, body after body
    F, T       (n_b, 3)   applied force and torque per body
    a, eta              blob radius and viscosity
    slip       (N, 3) or None   apparent slip per blob
    """

    q: np.ndarray
    theta: np.ndarray
    blob_start: np.ndarray
    rho: np.ndarray
    F: np.ndarray
    T: np.ndarray
    a: float
    eta: float = 1.0
    slip: np.ndarray | None = None
    name: str = ""

    @property
    def n_bodies(self) -> int:
        return int(self.q.shape[0])

    @property
    def n_blobs(self) -> int:
        return int(self.rho.shape[0])


class _CellGrid:
    """Uniform cell list over the (x, y) plane for rejection sampling."""

    def __init__(self, cell: float):
        self.cell = cell
        self.cells: dict = {}

    def key(self, p):
        return (int(math.floor(p[0] / self.cell)), int(math.floor(p[1] / self.cell)))

    def neighbours(self, p):
        cx, cy = self.key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                yield from self.cells.get((cx + dx, cy + dy), ())

    def add(self, idx, p):
        self.cells.setdefault(self.key(p), []).append(idx)


def _place(rng, radii, box, zlo, zhi, gap, rho_of=None, a=0.0, max_tries=2_000_000):
    """Random sequential placement of bodies with bounding radii `radii`.

    Centres are uniform in [0, box]^2 x [zlo, zhi]; two bodies are accepted
    only if their centres are at least r_p + r_q + gap apart.  When `rho_of`
    is given, each body's orientation is drawn as well and rejected unless
    every blob stays at height >= a.  A centre at least r_p + a above the
    wall keeps every blob at height >= a whatever the orientation, so the
    orientation test only runs below that height.
    """
    n = len(radii)
    cell = 2.0 * max(radii) + gap
    grid = _CellGrid(cell)
    centres = np.zeros((n, 3))
    placed = []  # (x, y, z, r) of accepted bodies, plain floats
    quats = random_unit_quaternions(rng, n)
    tries = 0
    for p in range(n):
        rp = float(radii[p])
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("placement did not converge; domain too dense")
            cx, cy, cz = rng.uniform(0, box), rng.uniform(0, box), rng.uniform(zlo, zhi)
            ok = True
            for k in grid.neighbours((cx, cy)):
                x, y, z, rk = placed[k]
                lim = rp + rk + gap
                if math.sqrt((cx - x) ** 2 + (cy - y) ** 2 + (cz - z) ** 2) < lim:
                    ok = False
                    break
            if not ok:
                continue
            if rho_of is not None and cz - rp < a:
                th = quats[p]
                if cz + _lowest_blob_height(th, rho_of(p)) < a:
                    quats[p] = random_unit_quaternions(rng, 1)[0]
                    continue
            centres[p] = (cx, cy, cz)
            placed.append((cx, cy, cz, rp))
            grid.add(p, (cx, cy))
            break
    return centres, quats


def sphere_suspension(
    seed: int,
    n_bodies: int,
    n_blobs: int,
    a: float,
    box: float,
    zlo: float,
    zhi: float,
    radius: float = 1.0,
    force_sigma: float = 0.1,
    torque_sigma: float = 0.1,
    gravity: float = 1.0,
    eta: float = 1.0,
    name: str = "",
) -> Suspension:
    """Identical icosahedral shells placed without overlap above the wall.

    Blobs on distinct bodies stay at least 2a apart (centre distance
    >= 2(R_g + a)); every blob stays at z >= a provided zlo - R_g >= a.
    F = (0, 0, -gravity) + N(0, force_sigma^2) per component,
    T = N(0, torque_sigma^2) per component.
    """
    rng = np.random.default_rng(seed)
    rho1 = shell(n_blobs, radius)
    if zlo - radius < a:
        raise ValueError("shell would reach below z = a")
    centres, quats = _place(rng, [radius] * n_bodies, box, zlo, zhi, 2.0 * a)
    F = rng.normal(0.0, force_sigma, (n_bodies, 3)) if force_sigma > 0 else np.zeros((n_bodies, 3))
    F[:, 2] -= gravity
    T = rng.normal(0.0, torque_sigma, (n_bodies, 3)) if torque_sigma > 0 else np.zeros((n_bodies, 3))
    return Suspension(
        q=centres,
        theta=quats,
        blob_start=np.arange(n_bodies + 1, dtype=np.int64) * n_blobs,
        rho=np.tile(rho1, (n_bodies, 1)),
        F=F,
        T=T,
        a=a,
        eta=eta,
        name=name,
    )


def mixed_suspension(
    seed: int,
    n_bodies: int,
    box: float | None = None,
    zlo: float = 1.2,
    zhi: float = 3.0,
    sphere_a: float = 0.243,
    boomerang_a: float = 0.1625,
    force_sigma: float = 0.1,
    torque_sigma: float = 0.1,
    eta: float = 1.0,
    name: str = "",
) -> Suspension:
    """Half 42-blob shells, half 15-blob boomerangs, random orientations.

    One blob radius serves the whole suspension (the mobility has a single
    a); it is the smaller of the two shape radii so that every body keeps its
    blobs at a/s <= 1/2.  The patch side defaults to sqrt(n_b / 0.04): half
    the body area density of 8 bodies per 10 x 10, because placement rejects
    on bounding spheres (boomerang bounding radius 1.64) and jams at the full
    density for hundreds of bodies.
    """
    rng = np.random.default_rng(seed)
    a = min(sphere_a, boomerang_a)
    if box is None:
        box = math.sqrt(n_bodies / 0.04)
    kinds = rng.integers(0, 2, n_bodies)  # 0 = sphere, 1 = boomerang
    sph = shell(42, 1.0)
    boo = boomerang15()
    shapes = [sph if k == 0 else boo for k in kinds]
    radii = [float(np.linalg.norm(s, axis=1).max()) for s in shapes]
    centres, quats = _place(
        rng, radii, box, zlo, zhi, 2.0 * a, rho_of=lambda p: shapes[p], a=a
    )
    counts = np.array([s.shape[0] for s in shapes], dtype=np.int64)
    blob_start = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    F = rng.normal(0.0, force_sigma, (n_bodies, 3))
    F[:, 2] -= 1.0
    T = rng.normal(0.0, torque_sigma, (n_bodies, 3))
    return Suspension(
        q=centres,
        theta=quats,
        blob_start=blob_start,
        rho=np.concatenate(shapes, axis=0),
        F=F,
        T=T,
        a=a,
        eta=eta,
        name=name,
    )


def blob_cloud(seed: int, n: int, a: float, box: float, zlo: float, zhi: float):
    """Free blobs: x, y ~ U[0, box], z ~ U[zlo, zhi], f ~ N(0, 1) per component.

    Returns (r, f), both (n, 3) float64.
    """
    rng = np.random.default_rng(seed)
    r = np.empty((n, 3))
    r[:, 0] = rng.uniform(0.0, box, n)
    r[:, 1] = rng.uniform(0.0, box, n)
    r[:, 2] = rng.uniform(zlo, zhi, n)
    f = rng.standard_normal((n, 3))
    return r, f


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------
def config_small_suspension(seed: int = 1) -> Suspension:
    """8 shells of 42 blobs (R_g = 1, a = 0.243), centres in [0,10]^2 x [1.5,4].

    N = 336 blobs; solved in FP64 to a relative residual of 1e-10.
    """
    return sphere_suspension(seed, 8, 42, 0.243, 10.0, 1.5, 4.0, name="8x42 shells, a=0.243")


def config_matvec_cloud(seed: int = 1, n: int = 65536):
    """N = 65,536 blobs, a = 0.5, x, y ~ U[0, 400], z ~ U[a, 3a], f ~ N(0, 1)."""
    a = 0.5
    r, f = blob_cloud(seed, n, a, 400.0, a, 3.0 * a)
    return r, f, a


def config_monolayer(seed: int = 1, n_bodies: int = 4096, box: float = 200.0) -> Suspension:
    """Sedimented monolayer: 162-blob shells (R_g = 1, a = 0.12) in a 200 x 200
    patch with centre heights in [1.2, 1.6]; gravity plus N(0, 0.1^2) torques.
    """
    return sphere_suspension(
        seed, n_bodies, 162, 0.12, box, 1.2, 1.6, force_sigma=0.0, torque_sigma=0.1,
        name=f"{n_bodies}x162 shells, a=0.12",
    )


def config_batched(seed: int = 1, n_problems: int = 256, lo: int = 8, hi: int = 2048):
    """Independent mixed suspensions with log-uniform body counts in [lo, hi]."""
    rng = np.random.default_rng(seed)
    counts = np.exp(rng.uniform(math.log(lo), math.log(hi), n_problems)).astype(int)
    return [mixed_suspension(int(seed * 100003 + i), int(c)) for i, c in enumerate(counts)]


def config_serving_request(seed: int, lo_blobs: int = 100, hi_blobs: int = 200_000) -> Suspension:
    """One serving request: a mixed suspension whose blob count is drawn
    log-uniformly in [lo_blobs, hi_blobs] (bodies average 28.5 blobs)."""
    rng = np.random.default_rng(seed)
    n_blobs = math.exp(rng.uniform(math.log(lo_blobs), math.log(hi_blobs)))
    n_bodies = max(1, int(round(n_blobs / 28.5)))
    return mixed_suspension(int(seed) * 7919 + 1, n_bodies)
