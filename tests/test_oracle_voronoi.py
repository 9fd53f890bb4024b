"""The Voronoi oracle (oracle/voronoi.py, the cell written out from its
definition, Sec. 2) pinned against closed forms and identities:

- a Cartesian lattice in a non-cubic box: every cell is the lattice box, its
  six faces have the known areas, centroids and volume;
- a triangular lattice in 2D: every cell is the regular hexagon of inradius
  a/2 (area sqrt(3)/2 a^2, six edges of length a/sqrt(3));
- random generators: the volumes fill the box, every face is found from both
  sides with the same area and the same centroid, and every cell is closed
  (sum of A n over its faces = 0, the divergence theorem).
A dropped or duplicated plane, a wrong image shift or a mis-signed normal
fails one of them."""
import numpy as np
import pytest

pytest.importorskip("scipy.spatial")

from harness import ics
from oracle import voronoi as OV


def test_cartesian_lattice_cells_are_boxes():
    box = np.array([1.0, 0.8, 1.2])
    n = 4
    pts, h = ics.lattice_nodes((n, n, n), box)
    faces, vol = OV.tessellate(pts, box)
    np.testing.assert_allclose(vol, np.prod(h), rtol=1e-12)
    areas = {0: h[1] * h[2], 1: h[0] * h[2], 2: h[0] * h[1]}
    for i, f in enumerate(faces):
        assert len(f) == 6
        for (j, *s), (a, c) in f.items():
            d = pts[j] + np.array(s) * box - pts[i]
            ax = int(np.argmax(np.abs(d)))
            assert abs(abs(d[ax]) - h[ax]) < 1e-12 and np.abs(np.delete(d, ax)).max() < 1e-12
            assert abs(a - areas[ax]) < 1e-12
            np.testing.assert_allclose(c, pts[i] + 0.5 * d, atol=1e-12)


def test_triangular_lattice_cells_are_hexagons():
    a, nx, ny = 0.1, 8, 6                       # ny even: the shifted rows close periodically
    dy = a * np.sqrt(3) / 2
    pts = np.array([[(x + 0.5 * (y % 2)) * a + 0.01, y * dy + 0.01] for y in range(ny) for x in range(nx)])
    box = np.array([nx * a, ny * dy])
    faces, vol = OV.tessellate(pts, box)
    np.testing.assert_allclose(vol, np.sqrt(3) / 2 * a * a, rtol=1e-12)
    for f in faces:
        assert len(f) == 6
        for (j, *s), (edge, c) in f.items():
            assert abs(edge - a / np.sqrt(3)) < 1e-12


@pytest.mark.parametrize("dim,n,seed", [(3, 60, 1), (2, 80, 2)])
def test_random_cells_fill_the_box_and_close(dim, n, seed):
    rng = np.random.default_rng(seed)
    box = np.array([1.0, 1.3, 0.9][:dim])
    pts = rng.uniform(0, 1, (n, dim)) * box
    faces, vol = OV.tessellate(pts, box)
    assert abs(vol.sum() - np.prod(box)) < 1e-12 * np.prod(box)
    for i, f in enumerate(faces):
        closure = np.zeros(dim)
        total = 0.0
        for (j, *s), (a, c) in f.items():
            d = pts[j] + np.array(s) * box - pts[i]
            closure += a * d / np.linalg.norm(d)
            total += a
            back = faces[j][(i,) + tuple(-v for v in s)]
            assert abs(back[0] - a) < 1e-10 * a
            np.testing.assert_allclose(back[1], c - np.array(s) * box, atol=1e-10)
        assert np.linalg.norm(closure) < 1e-10 * total
