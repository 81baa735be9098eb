"""Seeded synthetic inputs shaped like the workloads of arXiv 1612.04082.

This module is shared by the tests, the benchmark and the oracle's callers.  It holds
geometry and random numbers only -- none of the method's arithmetic (no kernel, no
quadrature, no tree): triangulated surfaces, point clouds on surfaces with their normals,
and random densities.  Everything is numpy, FP64, and reproducible from the seed.

Shapes follow the paper's benchmarks:
  * icosphere            -- sphere surfaces for the Lame closed-form tests;
  * voxel_surface        -- "each side of a cell on the boundary -> 4 triangles"
                            (Sec. "Performance and scalability": 24 N^2 triangles for an
                            N^3 cube), used for cubes, cantilever boxes and voxel masks;
  * box_with_voids_points -- points on a 2x1x1 box with spherical voids, the shape of
                            the surface point clouds the FMM sums over.
"""
from __future__ import annotations

import numpy as np

SEED_GEOMETRY = 1612
SEED_DENSITY = 4082
SEED_SUBSAMPLE = 7


# --------------------------------------------------------------------------- spheres
def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0), inward: bool = False):
    """Icosahedron subdivided `level` times, vertices projected onto the sphere.

    Returns (verts [nv,3] float64, tris [nt,3] int32), nt = 20 * 4**level.  Triangles
    are ordered so that the right-hand-rule normal points outward (inward if `inward`).
    """
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    T = np.array(faces, dtype=np.int32)
    # orient outward: check the sign of (n . (centroid - center)) per face
    c0 = np.asarray(center, dtype=np.float64)
    p0, p1, p2 = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    out = np.einsum("ij,ij->i", n, (p0 + p1 + p2) / 3.0 - c0) > 0
    T[~out] = T[~out][:, [0, 2, 1]]
    if inward:
        T = T[:, [0, 2, 1]].copy()
    return V, np.ascontiguousarray(T, dtype=np.int32)


# --------------------------------------------------------------------------- voxels
_FACE_DIRS = [(0, -1), (0, +1), (1, -1), (1, +1), (2, -1), (2, +1)]


def voxel_surface(mask: np.ndarray, h: float = 1.0, origin=(0.0, 0.0, 0.0)):
    """Boundary of the filled voxels of `mask` (bool [nx,ny,nz], cell size h).

    Every cell face between a filled cell and an empty cell (or the outside) becomes 4
    triangles fanned to the face centre, ordered so the normal points out of the
    material.  Returns (verts [nv,3], tris [nt,3] int32, face_cell [nt] int64 linear
    index of the owning filled cell, face_dir [nt] int8 in 0..5 = (-x,+x,-y,+y,-z,+z)).
    Corner vertices are shared between faces; face centres are per face.
    """
    m = np.asarray(mask, dtype=bool)
    nx, ny, nz = m.shape
    pad = np.zeros((nx + 2, ny + 2, nz + 2), dtype=bool)
    pad[1:-1, 1:-1, 1:-1] = m
    o = np.asarray(origin, dtype=np.float64)
    corner_ids = {}
    corners = []
    centers = []
    tri_list = []
    cell_list = []
    dir_list = []

    def corner(i, j, k):
        key = (i, j, k)
        idx = corner_ids.get(key)
        if idx is None:
            idx = len(corners)
            corner_ids[key] = idx
            corners.append((i, j, k))
        return idx

    # vectorised search for exposed faces, per direction
    for fd, (ax, sgn) in enumerate(_FACE_DIRS):
        shift = [0, 0, 0]
        shift[ax] = sgn
        nb = pad[1 + shift[0]:nx + 1 + shift[0], 1 + shift[1]:ny + 1 + shift[1],
                 1 + shift[2]:nz + 1 + shift[2]]
        ii, jj, kk = np.nonzero(m & ~nb)
        if ii.size == 0:
            continue
        # face corner offsets (in the two tangential axes), CCW seen from outside
        a1, a2 = [a for a in range(3) if a != ax]
        base = np.stack([ii, jj, kk], axis=1)
        if sgn > 0:
            base[:, ax] += 1
        quad = []
        for (u, v) in [(0, 0), (1, 0), (1, 1), (0, 1)]:
            c = base.copy()
            c[:, a1] += u
            c[:, a2] += v
            quad.append(c)
        # orientation: (e_a1 x e_a2) = +e_ax for the cyclic order; flip as needed
        cyc = (a2 - a1) % 3 == 1
        need_flip = (sgn > 0) != cyc
        lin = (ii * ny + jj) * nz + kk
        for f in range(ii.size):
            q = [corner(*quad[t][f]) for t in range(4)]
            if need_flip:
                q = q[::-1]
            cidx = len(centers)
            centers.append(0.25 * sum(np.asarray(quad[t][f], dtype=np.float64) for t in range(4)))
            for t in range(4):
                tri_list.append((-1 - cidx, q[t], q[(t + 1) % 4]))
                cell_list.append(lin[f])
                dir_list.append(fd)
    nc = len(corners)
    V = np.concatenate([np.asarray(corners, dtype=np.float64).reshape(-1, 3),
                        np.asarray(centers, dtype=np.float64).reshape(-1, 3)], axis=0) * h + o
    T = np.asarray(tri_list, dtype=np.int64).reshape(-1, 3)
    cm = T[:, 0] < 0
    T[cm, 0] = nc + (-1 - T[cm, 0])
    return (V, np.ascontiguousarray(T, dtype=np.int32), np.asarray(cell_list, dtype=np.int64),
            np.asarray(dir_list, dtype=np.int8))


def cube_mesh(n: int, size: float = 1.0, origin=(0.0, 0.0, 0.0)):
    """Boundary of an n^3 voxel cube of side `size`: 24 n^2 triangles."""
    v, t, _, _ = voxel_surface(np.ones((n, n, n), dtype=bool), size / n, origin)
    return v, t


def box_mesh(nx: int, ny: int, nz: int, h: float, origin=(0.0, 0.0, 0.0)):
    v, t, _, _ = voxel_surface(np.ones((nx, ny, nz), dtype=bool), h, origin)
    return v, t


def cantilever(n: int, patch_half: float = 0.25):
    """Cantilever 2x1x1 voxel box (cells 1/n, 40 n^2 triangles) with its boundary conditions:
    displacement 0 on the face x = 0, traction (0, 0, -1) on the x = 2 face elements whose
    centroids lie within patch_half of (y, z) = (0.5, 0.5), traction 0 elsewhere.
    Returns verts, tris, known_is_disp [nt, 3] uint8, values [nt, 3]."""
    v, t = box_mesh(2 * n, n, n, 1.0 / n)
    c = v[t].mean(axis=1)
    mask = np.zeros((len(t), 3), np.uint8)
    vals = np.zeros((len(t), 3))
    mask[c[:, 0] < 1e-9] = 1
    load = (c[:, 0] > 2 - 1e-9) & (np.abs(c[:, 1] - 0.5) <= patch_half) & (np.abs(c[:, 2] - 0.5) <= patch_half)
    vals[load] = [0.0, 0.0, -1.0]
    return v, t, mask, vals


def periodic_cell_voids(n: int = 128, n_voids: int | None = None, seed: int = SEED_GEOMETRY):
    """Unit periodic cell with 8-16 separate ellipsoidal voids (semi-axes U(0.04, 0.16),
    random rotations, inside the cell; bounding spheres at least 4 voxels apart, so every void
    surface is a closed manifold of its own), voxelised on an n^3 grid.  Returns the boundary
    of the void voxels as triangles (4 per exposed face) with normals pointing out of the
    material, i.e. into the voids: verts [nv, 3], tris [nt, 3] int32."""
    rng = np.random.default_rng(seed + 4)
    k = int(rng.integers(8, 17)) if n_voids is None else n_voids
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    void = np.zeros(len(P), bool)
    placed = []  # (centre, bounding radius)
    tries = 0
    while len(placed) < k:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place the voids")
        ax = rng.uniform(0.04, 0.16, 3)
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        m = ax.max() + 2 * h
        ctr = rng.uniform(m, 1 - m, 3)  # the void stays inside the cell
        if any(np.linalg.norm(ctr - c2) < m + m2 + 4 * h for c2, m2 in placed):
            continue
        placed.append((ctr, m))
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        L = (P - ctr) @ R / ax
        void |= np.einsum("ij,ij->i", L, L) <= 1.0
    mask = void.reshape(n, n, n)
    V, T, _, _ = voxel_surface(mask, h)
    return V, np.ascontiguousarray(T[:, [0, 2, 1]], dtype=np.int32)  # normals into the voids


# --------------------------------------------------------------------------- point clouds
def box_voids(n_voids: int = 20, box=(2.0, 1.0, 1.0), rmin=0.05, rmax=0.15, margin=0.05,
              seed: int = SEED_GEOMETRY):
    """Non-overlapping spheres inside the box, at least `margin` from its faces."""
    rng = np.random.default_rng(seed)
    B = np.asarray(box, dtype=np.float64)
    cs, rs = [], []
    tries = 0
    while len(cs) < n_voids:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place voids")
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(r + margin, B - r - margin)
        if all(np.linalg.norm(c - c2) > r + r2 + margin for c2, r2 in zip(cs, rs)):
            cs.append(c)
            rs.append(r)
    return np.array(cs), np.array(rs)


def box_with_voids_points(n: int, n_voids: int = 20, box=(2.0, 1.0, 1.0), seed: int = SEED_GEOMETRY):
    """`n` points area-uniform on the surface of [0,2]x[0,1]^2 with spherical voids.

    Returns (pts [n,3], nrm [n,3]) in float64; normals point out of the material (out of
    the box on its faces, into the void on a void's sphere).
    """
    B = np.asarray(box, dtype=np.float64)
    cs, rs = box_voids(n_voids, box, seed=seed)
    face_areas = np.array([B[1] * B[2]] * 2 + [B[0] * B[2]] * 2 + [B[0] * B[1]] * 2)
    sph_areas = 4.0 * np.pi * rs ** 2
    areas = np.concatenate([face_areas, sph_areas])
    rng = np.random.default_rng(seed + 1)
    which = rng.choice(areas.size, size=n, p=areas / areas.sum())
    pts = np.empty((n, 3))
    nrm = np.empty((n, 3))
    for f in range(6):
        sel = np.nonzero(which == f)[0]
        ax, side = f // 2, f % 2
        p = rng.uniform(0.0, 1.0, size=(sel.size, 3)) * B
        p[:, ax] = side * B[ax]
        nn = np.zeros((sel.size, 3))
        nn[:, ax] = 1.0 if side else -1.0
        pts[sel], nrm[sel] = p, nn
    for s in range(rs.size):
        sel = np.nonzero(which == 6 + s)[0]
        g = rng.normal(size=(sel.size, 3))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        pts[sel] = cs[s] + rs[s] * g
        nrm[sel] = -g
    return pts, nrm


def periodic_cell_points(n: int, n_voids: int = 12, lo=(0.0, 0.0, 0.0), side: float = 1.0,
                         seed: int = SEED_GEOMETRY):
    """`n` points area-uniform on the surfaces of `n_voids` non-overlapping spherical voids of a
    periodic cubic cell [lo, lo + side]^3 (radii U(0.05, 0.15) side, centres anywhere in the
    cell, distances measured across the cell's faces), wrapped into the cell: voids that cross a
    face appear in pieces on both sides, so the near field of a point near a face lies across it.

    Returns (pts [n,3], nrm [n,3]) in float64, normals into the voids.
    """
    rng = np.random.default_rng(seed + 11)
    lo = np.asarray(lo, dtype=np.float64)
    cs, rs = [], []
    tries = 0
    while len(cs) < n_voids:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place voids")
        r = rng.uniform(0.05, 0.15) * side
        c = rng.uniform(0.0, side, 3)
        ok = True
        for c2, r2 in zip(cs, rs):
            d = c - c2
            d -= side * np.round(d / side)  # nearest image
            ok &= np.linalg.norm(d) > r + r2 + 0.02 * side
        if ok:
            cs.append(c)
            rs.append(r)
    rs = np.array(rs)
    which = rng.choice(n_voids, size=n, p=rs ** 2 / (rs ** 2).sum())
    g = rng.normal(size=(n, 3))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    pts = np.array(cs)[which] + rs[which, None] * g
    return lo + np.mod(pts, side), -g


def surface_batch(n_sets: int = 32, lo: int = 5000, hi: int = 250000, seed: int = SEED_GEOMETRY):
    """A batch of independent box-with-voids surfaces of uneven size: set sizes log-uniform in
    [lo, hi], 4 to 19 voids each, each box scaled and placed on its own.

    Returns (pts [N,3], nrm [N,3], off [n_sets + 1]) with set k in rows off[k]:off[k+1].
    """
    rng = np.random.default_rng(seed + 7)
    sizes = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_sets)).astype(np.int64)
    pts, nrm = [], []
    for k, n in enumerate(sizes):
        x, nn = box_with_voids_points(int(n), n_voids=4 + k % 16, seed=seed + 100 + k)
        pts.append(x * rng.uniform(0.5, 2.0) + rng.uniform(-10.0, 10.0, size=3))
        nrm.append(nn)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(pts), np.concatenate(nrm), off


def densities(n: int, ncol: int = 1, seed: int = SEED_DENSITY):
    """Two N(0,1) 3-vector density arrays (single layer, double layer), [n, 3*ncol]."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 3 * ncol)), rng.normal(size=(n, 3 * ncol))


def subsample(n: int, k: int, seed: int = SEED_SUBSAMPLE):
    """k distinct indices in [0, n), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


def uniform_cloud(n: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), seed: int = SEED_GEOMETRY):
    """n points uniform in a box with random unit normals (volume-filling test cloud)."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, size=(n, 3))
    nn = rng.normal(size=(n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    return p, nn
