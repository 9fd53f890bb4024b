"""Pins of the host tessellator (input generator): closure, volumes, symmetry,
lattice degeneracies, thread independence, and agreement with qhull."""
import itertools

import numpy as np
import pytest

from harness import ics
from harness.tess import tessellate


def _closure(T):
    """sum_faces A n_out per cell; zero for a closed polytope (Gauss theorem)."""
    dim, n = T.dim, T.n_cells
    rL = T.points[T.cells[:, 0]]
    rR = T.points[T.cells[:, 1]] + T.shift * T.box
    d = rR - rL
    nrm = d / np.linalg.norm(d, axis=1)[:, None]
    acc = np.zeros((n, dim))
    np.add.at(acc, T.cells[:, 0], T.area[:, None] * nrm)
    np.add.at(acc, T.cells[:, 1], -T.area[:, None] * nrm)
    tot = np.zeros(n)
    np.add.at(tot, T.cells[:, 0], T.area)
    np.add.at(tot, T.cells[:, 1], T.area)
    return np.linalg.norm(acc, axis=1) / tot


@pytest.mark.parametrize("dim,n,jit", [(2, 24, 0.1), (3, 10, 0.2), (3, 12, 0.45)])
def test_closed_cells_and_total_volume(dim, n, jit):
    rng = np.random.default_rng(11)
    box = np.ones(dim) if dim == 3 else np.array([2.0, 1.0])
    dims = (n,) * dim if dim == 3 else (2 * n, n)
    pts = ics.jittered_lattice(dims, box, jit, rng)
    T = tessellate(pts, box)
    assert T.asymmetric == 0
    assert abs(T.volume.sum() - np.prod(box)) < 1e-12 * np.prod(box)
    assert _closure(T).max() < 1e-12
    # the face plane bisects the generators: centroid equidistant from both
    rL = T.points[T.cells[:, 0]]
    rR = T.points[T.cells[:, 1]] + T.shift * T.box
    dl = np.linalg.norm(T.centroid - rL, axis=1)
    dr = np.linalg.norm(T.centroid - rR, axis=1)
    assert np.max(np.abs(dl - dr) / np.linalg.norm(rR - rL, axis=1)) < 1e-10


def test_exact_lattice_drops_zero_area_faces():
    nodes, h = ics.lattice_nodes((6, 6, 6), np.ones(3))
    T = tessellate(nodes, np.ones(3))
    assert T.n_faces == 3 * 216                     # six faces per cube, each shared
    assert np.allclose(T.area, h[0] ** 2, rtol=1e-14)
    assert np.allclose(T.volume, h[0] ** 3, rtol=1e-14)
    nodes2, h2 = ics.lattice_nodes((8, 4), np.array([2.0, 1.0]))
    T2 = tessellate(nodes2, np.array([2.0, 1.0]))
    assert T2.n_faces == 2 * 32
    assert np.allclose(T2.area, 0.25, rtol=1e-14)


def test_thread_count_does_not_change_output():
    rng = np.random.default_rng(3)
    pts = ics.jittered_lattice((9, 9, 9), np.ones(3), 0.3, rng)
    a = tessellate(pts, np.ones(3), nthreads=1)
    b = tessellate(pts, np.ones(3), nthreads=5)
    for f in ("cells", "shift", "area", "centroid", "volume", "com"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def _qhull_faces(pts, box):
    """Voronoi faces of the central copy from scipy/qhull on 3^D periodic images."""
    sp = pytest.importorskip("scipy.spatial")
    dim = pts.shape[1]
    n = len(pts)
    imgs, ids, shifts = [], [], []
    for s in itertools.product((-1, 0, 1), repeat=dim):
        imgs.append(pts + np.array(s) * box)
        ids.append(np.arange(n))
        shifts.append(np.tile(s, (n, 1)))
    allp = np.concatenate(imgs)
    ids = np.concatenate(ids)
    shifts = np.concatenate(shifts)
    central = np.nonzero(np.all(shifts == 0, axis=1))[0]
    vor = sp.Voronoi(allp)
    faces = {}
    cset = set(central.tolist())
    for (a, b), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if a not in cset and b not in cset:
            continue
        if -1 in rv:
            continue
        if a not in cset:
            a, b = b, a
        verts = vor.vertices[rv]
        if dim == 2:
            area = np.linalg.norm(verts[1] - verts[0])
        else:
            # ridge vertices of a convex polygon, ordered by qhull around the ridge
            c = verts.mean(0)
            nrm = allp[b] - allp[a]
            nrm /= np.linalg.norm(nrm)
            u = np.cross(nrm, np.eye(3)[np.argmin(np.abs(nrm))])
            u /= np.linalg.norm(u)
            w = np.cross(nrm, u)
            ang = np.arctan2((verts - c) @ w, (verts - c) @ u)
            v = verts[np.argsort(ang)]
            area = 0.5 * np.linalg.norm(sum(np.cross(v[k], v[(k + 1) % len(v)]) for k in range(len(v))))
        if area < 1e-12:
            continue
        ds = shifts[b] - shifts[a]
        faces[(int(ids[a]), int(ids[b]), tuple(int(x) for x in ds))] = area
        faces[(int(ids[b]), int(ids[a]), tuple(-int(x) for x in ds))] = area
    return faces


@pytest.mark.parametrize("dim", [2, 3])
def test_matches_qhull(dim):
    rng = np.random.default_rng(5)
    box = np.ones(dim)
    dims = (7,) * dim
    pts = ics.jittered_lattice(dims, box, 0.35, rng)
    T = tessellate(pts, box)
    ref = _qhull_faces(pts, box)
    mine = {}
    for (L, R), s, a in zip(T.cells, T.shift, T.area):
        mine[(int(L), int(R), tuple(int(x) for x in s))] = a
        mine[(int(R), int(L), tuple(-int(x) for x in s))] = a
    assert set(mine) == set(ref)
    for k, a in ref.items():
        assert abs(mine[k] - a) <= 1e-9 * max(a, 1e-6), k
