"""Seeded synthetic inputs: tetrahedral unit-cell meshes and initial magnetisation.

This module is shared by the tests, the benchmark and the oracle's test drivers.  It
holds no arithmetic of the periodic micromagnetic method itself: it only produces
node coordinates (metres), tetrahedra (4 node indices each, positively oriented) and
unit magnetisation vectors, all from fixed seeds.

The workloads follow the geometries of the paper (Fig. 1 categories, Sec. 4.2-4.5):
a 2D-periodic film filling its cell (touching, non-protruding), a 3D lattice of
spheres (non-touching), and a 1D-periodic wire with bumps and a shear so that the
cell protrudes past its period (touching, protruding; Sec. 3.2, Eq. 18).
Periodic faces of every mesh conform: a node on a low face has a partner on the
opposite face displaced by exactly one period (up to rounding), as Eq. 5 requires.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh", "kuhn_box", "film_cell", "cube_cell", "prism_cell", "sphere_lattice",
    "wire_cell", "batch_cells", "granular_cell", "voronoi_grains", "m_tilted", "m_random", "m_vortex", "m_uniform", "net_init",
]


@dataclass
class Mesh:
    """A tetrahedral unit cell plus the periods it is meant to be used with."""
    xyz: np.ndarray            # (N, 3) float64, metres
    tets: np.ndarray           # (T, 4) int32, positively oriented
    periods: tuple             # (L1, L2, L3); 0 = not periodic along that axis
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def _orient(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Swap two vertices of every negatively oriented tetrahedron."""
    tets = np.ascontiguousarray(tets, dtype=np.int64)
    a = xyz[tets[:, 1]] - xyz[tets[:, 0]]
    b = xyz[tets[:, 2]] - xyz[tets[:, 0]]
    c = xyz[tets[:, 3]] - xyz[tets[:, 0]]
    det = np.einsum("ij,ij->i", a, np.cross(b, c))
    neg = det < 0
    tets[neg, 2], tets[neg, 3] = tets[neg, 3].copy(), tets[neg, 2].copy()
    return tets


def _volumes(xyz: np.ndarray, tets: np.ndarray) -> np.ndarray:
    a = xyz[tets[:, 1]] - xyz[tets[:, 0]]
    b = xyz[tets[:, 2]] - xyz[tets[:, 0]]
    c = xyz[tets[:, 3]] - xyz[tets[:, 0]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0


def kuhn_box(nx: int, ny: int, nz: int, h: float | tuple = 1e-9, origin=(0.0, 0.0, 0.0),
             jitter: float = 0.0, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Structured (nx x ny x nz) hexahedra, each split into 6 Kuhn tetrahedra.

    Every cube is cut along its main diagonal the same way, so shared faces, and
    opposite faces of the box, are split identically (conforming periodic faces).
    Nodes strictly inside the box (on no face) are moved by U(-jitter, jitter)*h
    per coordinate; nodes on faces keep their lattice positions.
    """
    hx, hy, hz = (h, h, h) if np.isscalar(h) else h
    i, j, k = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    i, j, k = i.transpose(2, 1, 0).ravel(), j.transpose(2, 1, 0).ravel(), k.transpose(2, 1, 0).ravel()
    xyz = np.stack([origin[0] + i * hx, origin[1] + j * hy, origin[2] + k * hz], axis=1).astype(np.float64)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        inside = (i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)
        d = rng.uniform(-jitter, jitter, size=(xyz.shape[0], 3)) * np.array([hx, hy, hz])
        xyz[inside] += d[inside]

    def nid(a, b, c):
        return a + (nx + 1) * (b + (ny + 1) * c)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.transpose(2, 1, 0).ravel(), cj.transpose(2, 1, 0).ravel(), ck.transpose(2, 1, 0).ravel()
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        p1 = unit[perm[0]]
        p2 = unit[perm[0]] + unit[perm[1]]
        v0 = nid(ci, cj, ck)
        v1 = nid(ci + p1[0], cj + p1[1], ck + p1[2])
        v2 = nid(ci + p2[0], cj + p2[1], ck + p2[2])
        v3 = nid(ci + 1, cj + 1, ck + 1)
        tets.append(np.stack([v0, v1, v2, v3], axis=1))
    tets = np.concatenate(tets, axis=0)
    # interleave so that the 6 tets of a cube are adjacent in memory
    tets = tets.reshape(6, -1, 4).transpose(1, 0, 2).reshape(-1, 4)
    tets = _orient(xyz, tets)
    vol = _volumes(xyz, tets)
    assert np.all(vol > 0), "kuhn_box produced a non-positive tetrahedron"
    return xyz, tets.astype(np.int32)


def film_cell(nx=20, ny=20, nz=2, h=1e-9, jitter=0.15, seed=0) -> Mesh:
    """Film filling a 2D-periodic (x, y) cell: (nx*h) x (ny*h) x (nz*h), z open."""
    xyz, tets = kuhn_box(nx, ny, nz, h, jitter=jitter, seed=seed)
    return Mesh(xyz, tets, (nx * h, ny * h, 0.0), name=f"film_{nx}x{ny}x{nz}")


def cube_cell(n=6, h=1e-9, jitter=0.15, seed=0) -> Mesh:
    """Cube filling a 3D-periodic cell (touching along all three axes)."""
    xyz, tets = kuhn_box(n, n, n, h, jitter=jitter, seed=seed)
    return Mesh(xyz, tets, (n * h, n * h, n * h), name=f"cube_{n}")


def prism_cell(nx=4, ny=4, nz=4, h=1e-9, jitter=0.15, seed=0) -> Mesh:
    """Square prism filling a 1D-periodic (z) cell; x and y are open."""
    xyz, tets = kuhn_box(nx, ny, nz, h, jitter=jitter, seed=seed)
    return Mesh(xyz, tets, (0.0, 0.0, nz * h), name=f"prism_{nx}x{ny}x{nz}")


@dataclass
class Grains:
    """Seeded grain structure of a cell: the grain of every tetrahedron, per-grain random
    orthonormal crystal axes (rows), anisotropy constants, and the exchange stiffness of every
    tetrahedron (A inside grains, A_iex in the boundary layer)."""
    tet_grain: np.ndarray     # (T,) int32
    axes: np.ndarray          # (G, 3, 3)
    K1: np.ndarray            # (G,) J/m^3
    Ku: np.ndarray            # (G,) J/m^3
    u: np.ndarray             # (G, 3) unit uniaxial axes
    A_tet: np.ndarray         # (T,) J/m


def granular_cell(n=8, h=1e-9, grains=6, K1=-4.5e3, Ku=0.0, A=1.3e-11, A_iex=0.2e-11, layer=0.6,
                  jitter=0.15, seed=0):
    """3D-periodic cube of n^3 Kuhn-split hexes with Voronoi grains of periodic seeds.

    A tetrahedron belongs to the grain of the seed nearest (periodically) to its centroid; it is
    in the boundary layer, with exchange stiffness A_iex, when the second-nearest seed is less
    than layer * h farther away than the nearest.  Crystal axes are seeded random orthonormal frames.
    Returns (Mesh, Grains)."""
    mesh = cube_cell(n, h=h, jitter=jitter, seed=seed)
    L = n * h
    rng = np.random.default_rng(seed + 101)
    seeds = rng.uniform(0, L, size=(grains, 3))
    cen = mesh.xyz[mesh.tets].mean(axis=1)
    d = cen[:, None, :] - seeds[None, :, :]
    d -= np.round(d / L) * L
    dist = np.linalg.norm(d, axis=2)
    order = np.argsort(dist, axis=1)
    tg = order[:, 0].astype(np.int32)
    gap = dist[np.arange(dist.shape[0]), order[:, 1]] - dist[np.arange(dist.shape[0]), order[:, 0]]
    A_tet = np.where(gap < layer * h, A_iex, A)
    axes = np.empty((grains, 3, 3))
    for g in range(grains):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        axes[g] = (q * np.sign(np.diag(r))[None, :]).T
    u = rng.normal(size=(grains, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    gr = Grains(tg, axes, np.full(grains, float(K1)), np.full(grains, float(Ku)), u, A_tet)
    return mesh, gr


def voronoi_grains(mesh: Mesh, grains: int, h: float, K1=-4.5e3, Ku=0.0, A=1.3e-11, A_iex=0.2e-11, layer=0.6,
                   seed=0) -> Grains:
    """Voronoi grains of seeded points over any mesh, periodic along its periodic axes: a
    tetrahedron belongs to the grain of the seed nearest (with the seeds' periodic images) to its
    centroid, and to the boundary layer (exchange stiffness A_iex) when the second-nearest seed is
    less than layer * h farther away.  Crystal axes are seeded random orthonormal frames."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed + 101)
    lo, hi = mesh.xyz.min(axis=0), mesh.xyz.max(axis=0)
    seeds = lo + rng.uniform(0, 1, size=(grains, 3)) * (hi - lo)
    shifts = [np.zeros(3)]
    for a in range(3):
        if mesh.periods[a] > 0:
            shifts = [s + d * mesh.periods[a] * np.eye(3)[a] for s in shifts for d in (-1, 0, 1)]
    pts = np.concatenate([seeds + s for s in shifts])
    owner = np.tile(np.arange(grains), len(shifts))
    cen = mesh.xyz[mesh.tets].mean(axis=1)
    dist, idx = cKDTree(pts).query(cen, k=2)
    tg = owner[idx[:, 0]].astype(np.int32)
    A_tet = np.where(dist[:, 1] - dist[:, 0] < layer * h, A_iex, A)
    axes = np.empty((grains, 3, 3))
    for g in range(grains):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        axes[g] = (q * np.sign(np.diag(r))[None, :]).T
    u = rng.normal(size=(grains, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return Grains(tg, axes, np.full(grains, float(K1)), np.full(grains, float(Ku)), u, A_tet)


def _fibonacci_sphere(n: int, R: float) -> np.ndarray:
    k = np.arange(n, dtype=np.float64) + 0.5
    phi = np.arccos(1.0 - 2.0 * k / n)
    theta = math.pi * (1.0 + math.sqrt(5.0)) * k
    return R * np.stack([np.cos(theta) * np.sin(phi), np.sin(theta) * np.sin(phi), np.cos(phi)], axis=1)


def _delaunay_tets(pts: np.ndarray, min_rel_vol: float) -> tuple[np.ndarray, np.ndarray]:
    from scipy.spatial import Delaunay
    tri = Delaunay(pts)
    tets = _orient(pts, tri.simplices)
    vol = _volumes(pts, tets)
    # drop flat slivers (vertices nearly coplanar), measured against edge length cubed
    e = np.linalg.norm(pts[tets[:, 1]] - pts[tets[:, 0]], axis=1)
    tets = tets[vol > min_rel_vol * e ** 3]
    used = np.unique(tets)
    remap = -np.ones(pts.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    return pts[used].copy(), remap[tets].astype(np.int32)


def sphere_lattice(L=50e-9, R=20e-9, h=None, target_nodes=200_000, seed=0) -> Mesh:
    """One sphere of radius R centred in a 3D-periodic cube of side L (non-touching).

    Nodes: a Fibonacci layer on the sphere surface at spacing h plus a jittered
    cubic lattice of spacing h inside (radius < R - h/2), then Delaunay.
    """
    if h is None:
        # solve (4/3 pi R^3)/h^3 + 4 pi R^2/h^2 ~ target for h
        f = lambda hh: (4.0 / 3.0) * math.pi * R ** 3 / hh ** 3 + 4 * math.pi * R ** 2 / hh ** 2 - target_nodes
        lo, hi = R / 1000, R
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if f(mid) > 0:
                lo = mid
            else:
                hi = mid
        h = 0.5 * (lo + hi)
    rng = np.random.default_rng(seed)
    n = int(math.ceil(R / h)) + 1
    g = np.arange(-n, n + 1, dtype=np.float64) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    P = P + rng.uniform(-0.15, 0.15, size=P.shape) * h
    P = P[np.linalg.norm(P, axis=1) < R - 0.5 * h]
    S = _fibonacci_sphere(int(round(4 * math.pi * R ** 2 / h ** 2)), R)
    pts = np.concatenate([S, P], axis=0) + L / 2
    xyz, tets = _delaunay_tets(pts, 1e-3)
    return Mesh(xyz, tets, (L, L, L), name="sphere_lattice", meta={"h": h, "R": R})


def wire_cell(L=100e-9, R=20e-9, target_nodes=1_000_000, seed=0, bumps=8, shear=0.15,
              grading=3.0, layers=None) -> Mesh:
    """1D-periodic (z) wire of radius R with Gaussian radial bumps and a shear.

    Cross-section: concentric rings whose spacing grows linearly 1:grading from the
    axis to the rim, triangulated by Delaunay; extruded in layers whose z spacing
    varies smoothly 1:grading along the period; every prism is split into three
    tetrahedra by the global-index rule so the z = 0 and z = L faces conform.
    Then nodes are pushed radially by 'bumps' seeded Gaussian bumps (3-6 nm high,
    5-10 nm wide, periodic in z) and sheared z' = z + shear * x, which makes the
    cell protrude past its period.
    """
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    # pick the centre spacing so that n2d * layers ~ target_nodes with layers ~ L / mean dz
    def ring_points(hc):
        pts = [np.zeros((1, 2))]
        r = 0.0
        radii = []
        while True:
            r = r + hc * (1.0 + (grading - 1.0) * r / R)
            if r > R - 0.3 * hc * grading:
                break
            radii.append(r)
        radii.append(R)
        for r in radii:
            hloc = hc * (1.0 + (grading - 1.0) * r / R)
            m = max(6, int(round(2 * math.pi * r / hloc)))
            t0 = rng.uniform(0, 2 * math.pi)
            t = t0 + 2 * math.pi * np.arange(m) / m
            pts.append(np.stack([r * np.cos(t), r * np.sin(t)], axis=1))
        return np.concatenate(pts, axis=0)

    def count(hc):
        # mean in-plane spacing ~ area-weighted; z spacing taken as the same mean
        nrm = 0
        r = 0.0
        while True:
            r = r + hc * (1.0 + (grading - 1.0) * r / R)
            if r > R:
                break
            nrm += max(6, int(round(2 * math.pi * r / (hc * (1.0 + (grading - 1.0) * r / R)))))
        mean_h = hc * (1.0 + grading) / 2.0
        return (nrm + 1) * max(4, int(round(L / mean_h)))

    lo, hi = R / 2000.0, R / 2.0
    for _ in range(60):
        mid = math.sqrt(lo * hi)
        if count(mid) > target_nodes:
            lo = mid
        else:
            hi = mid
    hc = math.sqrt(lo * hi)
    state = rng.bit_generator.state
    p2 = ring_points(hc)
    rng.bit_generator.state = state
    n2 = p2.shape[0]
    K = layers if layers is not None else max(4, int(round(target_nodes / n2)) - 1)
    tri = Delaunay(p2).simplices.astype(np.int64)
    # drop degenerate triangles (collinear points on a ring)
    a = p2[tri[:, 1]] - p2[tri[:, 0]]
    b = p2[tri[:, 2]] - p2[tri[:, 0]]
    area = 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    tri = tri[np.abs(area) > 1e-6 * hc * hc]
    tri = np.sort(tri, axis=1)
    # graded z layers: z(s) = L (s + a sin(2 pi s) / (2 pi)), dz ratio (1-a):(1+a) = 1:grading
    aa = (grading - 1.0) / (grading + 1.0)
    s = np.arange(K + 1, dtype=np.float64) / K
    zl = L * (s + aa * np.sin(2 * math.pi * s) / (2 * math.pi))
    zl[0], zl[K] = 0.0, L
    # bumps (periodic in z via the layer parameter s, so layer K equals layer 0)
    th_b = rng.uniform(0, 2 * math.pi, size=bumps)
    s_b = rng.uniform(0, 1, size=bumps)
    hgt = rng.uniform(3e-9, 6e-9, size=bumps)
    wid = rng.uniform(5e-9, 10e-9, size=bumps)
    rad = np.hypot(p2[:, 0], p2[:, 1])
    th = np.arctan2(p2[:, 1], p2[:, 0])
    xyz = np.empty(((K + 1) * n2, 3), dtype=np.float64)
    for j in range(K + 1):
        sj = s[j % K]
        disp = np.zeros(n2)
        for b_ in range(bumps):
            dth = np.angle(np.exp(1j * (th - th_b[b_])))
            dz = (sj - s_b[b_]) - np.round(sj - s_b[b_])
            disp += hgt[b_] * np.exp(-((dth * R) ** 2 + (dz * L) ** 2) / wid[b_] ** 2)
        scale = 1.0 + disp / R
        xyz[j * n2:(j + 1) * n2, 0] = p2[:, 0] * scale
        xyz[j * n2:(j + 1) * n2, 1] = p2[:, 1] * scale
        xyz[j * n2:(j + 1) * n2, 2] = zl[j]
    xyz[:, 2] = xyz[:, 2] + shear * xyz[:, 0]
    tets = []
    v0, v1, v2 = tri[:, 0], tri[:, 1], tri[:, 2]
    for j in range(K):
        b0, t0 = j * n2, (j + 1) * n2
        tets.append(np.stack([v0 + b0, v1 + b0, v2 + b0, v2 + t0], axis=1))
        tets.append(np.stack([v0 + b0, v1 + b0, v1 + t0, v2 + t0], axis=1))
        tets.append(np.stack([v0 + b0, v0 + t0, v1 + t0, v2 + t0], axis=1))
    tets = np.concatenate(tets, axis=0)
    # order tets layer-major, triangle-minor (spatially coherent)
    tets = tets.reshape(K, 3, -1, 4).transpose(0, 2, 1, 3).reshape(-1, 4)
    tets = _orient(xyz, tets)
    assert np.all(_volumes(xyz, tets) > 0), "wire_cell produced a non-positive tetrahedron"
    return Mesh(xyz, tets.astype(np.int32), (0.0, 0.0, L), name="wire",
                meta={"n2d": n2, "layers": K, "hc": hc})


def batch_cells(n_cells=64, seed=0, n_min=5000, n_max=80000, scale=1.0):
    """Independent 2D-periodic film or dot cells of uneven node counts.

    Cell i: thickness U(2, 10) nm, square period U(40, 200) nm, type film
    (fills the cell) or dot (disk of diameter U(0.6, 0.9) * period) with
    probability 1/2 each, node count ~ U{n_min..n_max} * scale.
    """
    rng = np.random.default_rng(seed)
    cells = []
    for i in range(n_cells):
        t = rng.uniform(2e-9, 10e-9)
        P = rng.uniform(40e-9, 200e-9)
        kind = "film" if rng.uniform() < 0.5 else "dot"
        n_target = int(rng.integers(n_min, n_max + 1) * scale)
        if kind == "film":
            # largest nx with (nx + 1)^2 (nz + 1) <= n_target, nz = max(1, round(t / (P / nx)))
            def film_nodes(k):
                return (k + 1) ** 2 * (max(1, int(round(t / (P / k)))) + 1)
            nx = 4
            while film_nodes(nx + 1) <= n_target:
                nx += 1
            hxy = P / nx
            nz = max(1, int(round(t / hxy)))
            xyz, tets = kuhn_box(nx, nx, nz, (hxy, hxy, t / nz), jitter=0.1, seed=seed * 1000 + i)
            cells.append(Mesh(xyz, tets, (P, P, 0.0), name=f"film{i}", meta={"kind": kind, "t": t}))
        else:
            D = rng.uniform(0.6, 0.9) * P
            cells.append(_dot_cell(D / 2, t, P, n_target, seed * 1000 + i))
    return cells


def _dot_cell(r, t, P, n_target, seed):
    """Disk (radius r, thickness t) centred in a square 2D-periodic cell of side P."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    # layers nz+1, in-plane spacing h: (pi r^2 / (0.866 h^2)) * (nz + 1) ~ n_target; the
    # count falls as h grows, so bisect on log h
    def count(h):
        return math.pi * r * r / (0.866 * h * h) * (max(1, int(round(t / h))) + 1)
    lo, hi = math.log(r * 1e-3), math.log(r)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if count(math.exp(mid)) > n_target:
            lo = mid
        else:
            hi = mid
    h = math.exp(hi)
    nz = max(1, int(round(t / h)))
    pts = [np.zeros((1, 2))]
    nr = max(1, int(round(r / h)))
    for k in range(1, nr + 1):
        rr = r * k / nr
        m = max(6, int(round(2 * math.pi * rr / h)))
        tt = rng.uniform(0, 2 * math.pi) + 2 * math.pi * np.arange(m) / m
        pts.append(np.stack([rr * np.cos(tt), rr * np.sin(tt)], axis=1))
    p2 = np.concatenate(pts)
    n2 = p2.shape[0]
    tri = np.sort(Delaunay(p2).simplices.astype(np.int64), axis=1)
    a = p2[tri[:, 1]] - p2[tri[:, 0]]
    b = p2[tri[:, 2]] - p2[tri[:, 0]]
    tri = tri[np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]) > 1e-6 * h * h]
    xyz = np.empty(((nz + 1) * n2, 3))
    for j in range(nz + 1):
        xyz[j * n2:(j + 1) * n2, :2] = p2 + P / 2
        xyz[j * n2:(j + 1) * n2, 2] = t * j / nz
    v0, v1, v2 = tri[:, 0], tri[:, 1], tri[:, 2]
    tets = []
    for j in range(nz):
        b0, t0 = j * n2, (j + 1) * n2
        tets += [np.stack([v0 + b0, v1 + b0, v2 + b0, v2 + t0], 1),
                 np.stack([v0 + b0, v1 + b0, v1 + t0, v2 + t0], 1),
                 np.stack([v0 + b0, v0 + t0, v1 + t0, v2 + t0], 1)]
    tets = _orient(xyz, np.concatenate(tets))
    return Mesh(xyz, tets.astype(np.int32), (P, P, 0.0), name="dot", meta={"kind": "dot", "t": t})


# ----------------------------------------------------------------------------------
# initial magnetisation (unit vectors), one per row of the given positions
# ----------------------------------------------------------------------------------

def m_uniform(n: int, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    return np.tile(d / np.linalg.norm(d), (n, 1))


def m_tilted(n: int, polar_deg: float = 5.0, seed: int = 1) -> np.ndarray:
    """+z tilted by exactly polar_deg with a seeded U[0, 2 pi) azimuth per row."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2 * math.pi, size=n)
    th = math.radians(polar_deg)
    return np.stack([math.sin(th) * np.cos(ph), math.sin(th) * np.sin(ph),
                     np.full(n, math.cos(th))], axis=1)


def m_random(n: int, seed: int = 1) -> np.ndarray:
    """Uniform random directions on the unit sphere."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def m_vortex(xyz: np.ndarray, core: float = 5e-9, centre=(0.0, 0.0)) -> np.ndarray:
    """Vortex about the z axis: m_z = exp(-(rho/core)^2), in-plane part circulating."""
    x = xyz[:, 0] - centre[0]
    y = xyz[:, 1] - centre[1]
    rho = np.hypot(x, y)
    mz = np.exp(-(rho / core) ** 2)
    inp = np.sqrt(np.clip(1.0 - mz * mz, 0.0, None))
    safe = np.where(rho > 0, rho, 1.0)
    return np.stack([-y / safe * inp, x / safe * inp, mz], axis=1)


# ----------------------------------------------------------------------------------
# initial weights of the surrogate network (seeded random numbers, passed in as inputs)
# ----------------------------------------------------------------------------------

def net_init(channels: int = 32, seed: int = 0) -> np.ndarray:
    """He-normal weights (variance 2 / fan_in, fan_in = 27 ci) and zero biases of the four
    3x3x3 layers 1 -> C -> C -> C -> 1, flattened layer by layer as W[co][ci][dz][dy][dx]
    followed by b[co] (float32)."""
    rng = np.random.default_rng(seed)
    out = []
    for co, ci in ((channels, 1), (channels, channels), (channels, channels), (1, channels)):
        out.append(rng.normal(0.0, math.sqrt(2.0 / (27 * ci)), size=co * ci * 27))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)
