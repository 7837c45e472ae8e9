"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds geometry and sampling only -- none of the method's arithmetic -- so that the
CUDA path and the CPU oracle can be fed identical inputs without sharing any code.

The paper evaluates surface samples of meshes rescaled into [-1, 1]^3 (Sec. 4.1), on 100^3
grids, random query sets and 1000^2 slice planes (Sec. 4.2, 4.3). Its meshes are not available,
so unions of random ellipsoids and boxes stand in for them: area-uniform samples with area
weights and outward normals, exactly the inputs winding numbers and smooth distances need.

Generators use numpy's PCG64 with a caller-given seed.
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 2506_02219


@dataclasses.dataclass
class Workload:
    """One evaluation problem: sources (points, weights, optional normals) and queries."""
    name: str
    points: np.ndarray            # [M, 3] float32
    weights: np.ndarray           # [M] float32, > 0
    normals: np.ndarray | None    # [M, 3] float32 unit vectors, or None
    queries: np.ndarray           # [N, 3] float32
    kernel: str                   # "coulomb" | "winding" | "smoothdist"
    softening: float = 1e-3
    alpha: float = 200.0
    leaf_size: int = 1
    S: int = 1


# ---------------------------------------------------------------------------------------------
# query sets
# ---------------------------------------------------------------------------------------------
def grid_plane(nx: int, ny: int, lo=(0.0, 0.0), hi=(1.0, 1.0), z: float = 0.5) -> np.ndarray:
    """Cell-centred nx x ny grid on the plane z = const, x fastest."""
    xs = lo[0] + (np.arange(nx) + 0.5) * (hi[0] - lo[0]) / nx
    ys = lo[1] + (np.arange(ny) + 0.5) * (hi[1] - lo[1]) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    q = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
    return q.astype(np.float32)


def grid_box(n: int, lo, hi) -> np.ndarray:
    """Cell-centred n^3 grid in the box [lo, hi], x fastest, then y, then z."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    axes = [lo[a] + (np.arange(n) + 0.5) * (hi[a] - lo[a]) / n for a in range(3)]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float32)


def uniform_box(n: int, lo, hi, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return (lo + rng.random((n, 3)) * (hi - lo)).astype(np.float32)


# ---------------------------------------------------------------------------------------------
# source sets
# ---------------------------------------------------------------------------------------------
def uniform_cube(n: int, seed: int, mass_lo: float = 0.5, mass_hi: float = 1.5):
    """n points uniform in the unit cube with masses U(mass_lo, mass_hi)."""
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3)).astype(np.float32)
    m = rng.uniform(mass_lo, mass_hi, n).astype(np.float32)
    return p, m


def _random_rotation(rng) -> np.ndarray:
    # uniform random rotation from a normalised Gaussian quaternion
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def ellipsoid_area(axes) -> float:
    """Surface area of an ellipsoid with semi-axes (a, b, c) by FP64 Gauss-Legendre quadrature of
    abc * |grad| over the unit sphere (cos(theta) nodes x uniform phi)."""
    a, b, c = (float(v) for v in axes)
    xg, wg = np.polynomial.legendre.leggauss(96)
    nphi = 192
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct = xg[:, None]
    st = np.sqrt(1 - ct * ct)
    ux, uy, uz = st * np.cos(phi)[None, :], st * np.sin(phi)[None, :], np.broadcast_to(ct, (96, nphi))
    g = a * b * c * np.sqrt((ux / a) ** 2 + (uy / b) ** 2 + (uz / c) ** 2)
    return float(np.sum(wg[:, None] * g) * (2 * np.pi / nphi))


class _Ellipsoid:
    def __init__(self, center, axes, rot):
        self.c = np.asarray(center, np.float64)
        self.ax = np.asarray(axes, np.float64)
        self.R = np.asarray(rot, np.float64)
        self.area = ellipsoid_area(self.ax)

    def inside(self, p):  # strictly inside
        loc = (p - self.c) @ self.R
        return np.sum((loc / self.ax) ** 2, axis=1) < 1.0

    def sample(self, rng, n):
        """n area-uniform surface points with outward normals: uniform sphere points mapped onto
        the ellipsoid, accepted with probability proportional to the area stretch."""
        a, b, c = self.ax
        gmax = max(1 / a, 1 / b, 1 / c)
        out_p, out_n = [], []
        need = n
        while need > 0:
            m = max(2 * need, 1024)
            u = rng.normal(size=(m, 3))
            u /= np.linalg.norm(u, axis=1, keepdims=True)
            g = np.sqrt((u[:, 0] / a) ** 2 + (u[:, 1] / b) ** 2 + (u[:, 2] / c) ** 2)
            keep = rng.random(m) < g / gmax
            u = u[keep][:need]
            loc = u * self.ax
            nrm = loc / self.ax ** 2
            nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
            out_p.append(loc @ self.R.T + self.c)
            out_n.append(nrm @ self.R.T)
            need -= u.shape[0]
        return np.concatenate(out_p), np.concatenate(out_n)


class _Box:
    def __init__(self, center, half):
        self.c = np.asarray(center, np.float64)
        self.h = np.asarray(half, np.float64)
        hx, hy, hz = self.h
        self.face_area = np.array([hy * hz, hy * hz, hx * hz, hx * hz, hx * hy, hx * hy]) * 4.0
        self.area = float(self.face_area.sum())

    def inside(self, p):
        return np.all(np.abs(p - self.c) < self.h, axis=1)

    def sample(self, rng, n):
        face = rng.choice(6, size=n, p=self.face_area / self.area)
        uv = rng.random((n, 3)) * 2 - 1
        axis = face // 2
        sign = np.where(face % 2 == 0, -1.0, 1.0)
        uv[np.arange(n), axis] = sign
        nrm = np.zeros((n, 3))
        nrm[np.arange(n), axis] = sign
        return uv * self.h + self.c, nrm


def shape_union(n: int, seed: int, n_ellipsoids: int = 8, n_boxes: int = 0, rescale: bool = True,
                heavy_fraction: float = 0.0, heavy_factor: float = 5.0):
    """n area-uniform samples on the surface of a union of random ellipsoids (centres
    U[-0.6, 0.6]^3, semi-axes U[0.15, 0.5], random rotations) and axis-aligned boxes (centres
    U[-0.6, 0.6]^3, half-extents U[0.1, 0.4]). Candidates are drawn on each shape in proportion
    to its area, those inside another shape are dropped, until n remain. Each sample carries the
    area weight A_i / N_i (shape area over candidates drawn on that shape) and its outward normal.
    With rescale, the set is scaled isotropically to fit [-1, 1]^3. heavy_fraction > 0 multiplies
    the weights of that fraction of the samples (a seeded random subset) by heavy_factor: a few
    heavier sources among uniform ones, as the paper's teaser scene has."""
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(n_ellipsoids):
        shapes.append(_Ellipsoid(rng.uniform(-0.6, 0.6, 3), rng.uniform(0.15, 0.5, 3), _random_rotation(rng)))
    for _ in range(n_boxes):
        shapes.append(_Box(rng.uniform(-0.6, 0.6, 3), rng.uniform(0.1, 0.4, 3)))
    areas = np.array([s.area for s in shapes])
    drawn = np.zeros(len(shapes), np.int64)
    pts, nrms, owner = [], [], []
    kept = 0
    while kept < n:
        batch = max(int((n - kept) * 1.3), 4096)
        counts = rng.multinomial(batch, areas / areas.sum())
        for i, s in enumerate(shapes):
            if counts[i] == 0:
                continue
            p, nv = s.sample(rng, int(counts[i]))
            drawn[i] += counts[i]
            outside = np.ones(p.shape[0], bool)
            for j, o in enumerate(shapes):
                if j != i:
                    outside &= ~o.inside(p)
            pts.append(p[outside]); nrms.append(nv[outside]); owner.append(np.full(int(outside.sum()), i))
            kept += int(outside.sum())
    P = np.concatenate(pts)
    Nv = np.concatenate(nrms)
    own = np.concatenate(owner)
    # random order, then keep exactly n (the drop is uniform over candidates, so weights stay valid)
    order = rng.permutation(P.shape[0])[:n]
    P, Nv, own = P[order], Nv[order], own[order]
    drawn_total = drawn.astype(np.float64) * (n / float(kept))  # candidates behind the kept subset
    w = areas[own] / drawn_total[own]
    if rescale:
        lo, hi = P.min(axis=0), P.max(axis=0)
        ctr = 0.5 * (lo + hi)
        s = 2.0 / float(np.max(hi - lo)) * 0.999
        P = (P - ctr) * s
        w = w * s * s
    if heavy_fraction > 0.0:
        heavy = np.random.default_rng(seed + 7).permutation(n)[: int(round(heavy_fraction * n))]
        w = w.copy()
        w[heavy] *= heavy_factor
    return P.astype(np.float32), w.astype(np.float32), Nv.astype(np.float32)


def bounding_box(points: np.ndarray):
    return points.min(axis=0).astype(np.float64), points.max(axis=0).astype(np.float64)


# ---------------------------------------------------------------------------------------------
# the named workloads
# ---------------------------------------------------------------------------------------------
def coulomb_cube(n_sources: int = 4096, grid: int = 64, seed: int = BASE_SEED + 0) -> Workload:
    """1/r potential, sources uniform in the unit cube with masses U(0.5, 1.5), softening 1e-3,
    queries on a grid x grid cell-centred grid over the plane z = 0.5, leaf size 1, S = 1."""
    p, m = uniform_cube(n_sources, seed)
    q = grid_plane(grid, grid, (0.0, 0.0), (1.0, 1.0), 0.5)
    return Workload("coulomb_cube_4096src_64x64plane", p, m, None, q, "coulomb", softening=1e-3)


def winding_ellipsoids(n_sources: int = 1 << 20, grid: int = 256, seed: int = BASE_SEED + 1) -> Workload:
    """Winding number of oriented area-weighted samples on a union of 8 random ellipsoids,
    queries on a grid^3 cell-centred grid over the sources' bounding box."""
    p, w, nv = shape_union(n_sources, seed, n_ellipsoids=8, n_boxes=0)
    lo, hi = bounding_box(p)
    q = grid_box(grid, lo, hi)
    return Workload(f"winding_8ellipsoids_{n_sources}src_{grid}cube", p, w, nv, q, "winding")


def winding_ellipsoids_random(n_sources: int = 1 << 20, n_queries: int = 1 << 24,
                              seed: int = BASE_SEED + 1) -> Workload:
    """The sources of winding_ellipsoids with as many queries drawn uniformly at random in their
    bounding box, in the order drawn (no spatial coherence between neighbouring queries: the
    random query sets of the paper's Fig. 4)."""
    p, w, nv = shape_union(n_sources, seed, n_ellipsoids=8, n_boxes=0)
    lo, hi = bounding_box(p)
    q = uniform_box(n_queries, lo, hi, seed + 11)
    return Workload(f"winding_8ellipsoids_{n_sources}src_{n_queries}random", p, w, nv, q, "winding")


def slice_plane_shapes(n_sources: int = 1 << 22, res: int = 1000, kernel: str = "smoothdist",
                       seed: int = BASE_SEED + 2, shuffle: bool = True) -> Workload:
    """Samples on a union of 8 random ellipsoids and 4 boxes, queries on a res x res slice plane
    z = 0 over [-1, 1]^2 (shuffled). Smooth distance (alpha = 200, unit weights) or Coulomb
    (area weights)."""
    p, w, nv = shape_union(n_sources, seed, n_ellipsoids=8, n_boxes=4)
    q = grid_plane(res, res, (-1.0, -1.0), (1.0, 1.0), 0.0)
    if shuffle:
        q = q[np.random.default_rng(seed + 7).permutation(q.shape[0])]
    if kernel == "smoothdist":
        w = np.ones_like(w)
    return Workload(f"{kernel}_shapes_{n_sources}src_{res}x{res}plane", p, w, nv, q, kernel, alpha=200.0)


def far_field_coulomb(n_sources: int = 1 << 20, res: int = 170, seed: int = BASE_SEED + 1) -> Workload:
    """The geometry of winding_ellipsoids (2^20 area-weighted samples, rescaled into [-1, 1]^3) with
    the Coulomb kernel, queried in empty space around it: the nodes of a res^3 grid over [-3, 3]^3
    that lie outside [-1.2, 1.2]^3 (the regime where most sources are far from every query)."""
    p, w, nv = shape_union(n_sources, seed, n_ellipsoids=8, n_boxes=0)
    g = np.linspace(-3.0, 3.0, res, dtype=np.float32)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    q = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    q = np.ascontiguousarray(q[np.abs(q).max(1) > 1.2], dtype=np.float32)
    return Workload(f"far_field_coulomb_{n_sources}src_{q.shape[0]}q", p, w, nv, q, "coulomb")


def sphere_fibonacci(n: int, radius: float = 1.0):
    """n Fibonacci-lattice points on a sphere with equal area weights and outward normals."""
    i = np.arange(n, dtype=np.float64) + 0.5
    z = 1 - 2 * i / n
    r = np.sqrt(1 - z * z)
    phi = i * np.pi * (3 - np.sqrt(5))
    nv = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    w = np.full(n, 4 * np.pi * radius * radius / n)
    return (nv * radius).astype(np.float32), w.astype(np.float32), nv.astype(np.float32)
