"""Host side of the optimisation procedure (Sec. "Parallel optimization procedure"): the
native voxel-surface extraction, the threshold update D_C = D_min + C (D_max - D_min) and
the post-processing, checked against the seeded numpy generator and against properties
fixed by geometry (closed, outward-oriented surfaces; the face count of Sec. "Performance
and scalability")."""
import numpy as np
import pytest

import workloads as W

K = pytest.importorskip("paper_1612_04082_gb300")


def random_mask(shape, seed, fill=0.6):
    return (np.random.default_rng(seed).random(shape) < fill).astype(np.uint8)


@pytest.mark.parametrize("shape,seed", [((5, 4, 3), 0), ((7, 2, 6), 1), ((1, 1, 1), 2), ((6, 6, 6), 3)])
def test_surface_matches_generator(shape, seed):
    m = random_mask(shape, seed)
    m.flat[0] = 1
    a = W.voxel_surface(m.astype(bool), 0.25, (0.5, -1.0, 2.0))
    b = K.voxel_surface(m, 0.25, (0.5, -1.0, 2.0))
    assert np.allclose(a[0], b[0], rtol=0, atol=1e-15)
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n", [1, 2, 5])
def test_cube_face_count_and_closed_outward(n):
    h = 1.0 / n
    V, T, cell, fdir = K.voxel_surface(np.ones((n, n, n), np.uint8), h)
    assert len(T) == 24 * n * n
    # every directed edge appears once and its reverse once: closed and consistently oriented
    e = np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]])
    fwd = set(map(tuple, e))
    assert len(fwd) == len(e) and all((b, a) in fwd for a, b in fwd)
    # divergence theorem: signed volume = enclosed volume (normals out of the material)
    vol = np.einsum("ij,ij->i", V[T[:, 0]], np.cross(V[T[:, 1]], V[T[:, 2]])).sum() / 6
    assert vol == pytest.approx(1.0, rel=1e-12)


def test_random_solid_signed_volume():
    m = random_mask((6, 5, 4), 7, 0.7)
    h = 0.3
    V, T, cell, fdir = K.voxel_surface(m, h)
    vol = np.einsum("ij,ij->i", V[T[:, 0]], np.cross(V[T[:, 1]], V[T[:, 2]])).sum() / 6
    assert vol == pytest.approx(m.sum() * h ** 3, rel=1e-12)
    # each face's owning voxel is material and its neighbour across the face is not
    d = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]])
    ijk = np.stack(np.unravel_index(cell, m.shape), 1)
    assert m[tuple(ijk.T)].all()
    nb = ijk + d[fdir]
    inside = ((nb >= 0) & (nb < np.array(m.shape))).all(1)
    assert not m[tuple(nb[inside].T)].any()


def test_threshold_rule():
    m = np.ones((4, 3, 2), np.uint8)
    td = np.arange(m.size, dtype=np.float32)  # D_min = 0, D_max = 23
    frozen = np.zeros_like(m)
    frozen.flat[1] = 1
    mm = m.copy()
    assert K.voxel_threshold(mm, td, 0.0, frozen) == 0
    mm = m.copy()
    n = K.voxel_threshold(mm, td, 0.25, frozen)  # D_C = 5.75: cells 0..5 below, cell 1 frozen
    assert n == 5 and mm.flat[1] == 1 and not mm.flat[[0, 2, 3, 4, 5]].any() and mm.flat[6:].all()
    # void cells do not enter the range
    mm = m.copy()
    mm.flat[:12] = 0
    n = K.voxel_threshold(mm, td, 0.5, None)  # range 12..23, D_C = 17.5
    assert n == 6 and mm.flat[18:].all() and not mm.flat[:18].any()
    with pytest.raises(K.KfmmError):
        K.voxel_threshold(m.copy(), td, 1.5)


def test_clean_isolated_and_disconnected():
    m = np.zeros((6, 3, 3), np.uint8)
    m[0:2, :, :] = 1        # block touching the support
    m[4, 1, 1] = 1          # isolated voxel
    m[5, 0, 0] = m[5, 0, 1] = 1  # small blob not connected to the support
    support = np.zeros_like(m)
    support[0, :, :] = 1
    mm = m.copy()
    n = K.voxel_clean(mm, support)
    assert n == 3 and mm[0:2].all() and mm[2:].sum() == 0
    mm = m.copy()  # without supports only the isolated voxel goes
    assert K.voxel_clean(mm, None) == 1 and mm[5, 0, 0] == 1 and mm[4, 1, 1] == 0
    keep = np.zeros_like(m)  # kept voxels survive both rules
    keep[4, 1, 1] = keep[5, 0, 0] = 1
    mm = m.copy()
    assert K.voxel_clean(mm, support, keep) == 1 and mm[4, 1, 1] == 1 and mm[5, 0, 0] == 1 and mm[5, 0, 1] == 0


@pytest.mark.parametrize("shape,seed", [((6, 6, 6), 4), ((5, 7, 4), 5)])
def test_periodic_surface_faces_and_orientation(shape, seed):
    """The periodic surface has one face (4 triangles) per material voxel face whose wrapped
    neighbour is void, with the normal out of the material (face_dir), none elsewhere; its
    oriented area sums to zero (closed on the torus); rolling the pattern across the cell's
    faces changes neither the face count nor the area."""
    m = random_mask(shape, seed, fill=0.7)
    h = 0.1
    V, T, cell, fdir = K.voxel_surface(m, h, periodic=True)
    expect = 0
    for ax in range(3):
        for sgn in (-1, 1):
            nb = np.roll(m, -sgn, axis=ax)  # the neighbour at index + sgn, wrapped
            expect += int(((m == 1) & (nb == 0)).sum())
    assert len(T) == 4 * expect
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(b - a, c - a)
    dirs = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]])
    assert np.all(np.einsum("ij,ij->i", cr, dirs[fdir]) > 0)
    assert np.abs(0.5 * cr.sum(axis=0)).max() < 1e-12
    area = 0.5 * np.linalg.norm(cr, axis=1).sum()
    lo, hi = V.min(axis=0), V.max(axis=0)
    assert np.all(lo >= -1e-15) and np.all(hi <= np.array(shape) * h + 1e-15)
    r = np.roll(m, (2, -1, 3), axis=(0, 1, 2))
    V2, T2, _, _ = K.voxel_surface(r, h, periodic=True)
    a2 = 0.5 * np.linalg.norm(np.cross(V2[T2[:, 1]] - V2[T2[:, 0]], V2[T2[:, 2]] - V2[T2[:, 0]]), axis=1).sum()
    assert len(T2) == len(T) and a2 == pytest.approx(area, rel=1e-12)
    # all material: no surface at all
    V3, T3, _, _ = K.voxel_surface(np.ones(shape, np.uint8), h, periodic=True)
    assert len(T3) == 0
