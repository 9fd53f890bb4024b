"""Voronoi cells of a periodic box written out from their definition (Sec. 2).

TEST INFRASTRUCTURE ONLY: tests/ compare the GPU mesh builder with it; the
CUDA path never uses it.

The cell of generator r_i is the set of points nearer to r_i than to any other
generator or periodic image of one: the intersection of the half-spaces
n.x <= h bounded by the bisectors, with n = r_j' - r_i and h = |n|^2 / 2 in
coordinates about r_i.  Here every image r_j + s L with s in {-1, 0, 1}^dim
enters (nothing is pruned), scipy's HalfspaceIntersection (a library
primitive) gives the cell's vertices, and a face is the set of vertices lying
on a bisector plane: its area and centroid are summed over a fan about the
vertex average in angular order (3D) or taken as a segment (2D).  Faces below
area_tol times the mean spacing to the power dim - 1 are dropped.

Output per cell: {(j, s): (area, centroid)} with the centroid absolute, in the
frame of cell i, and the cell volume from the divergence theorem,
V = sum_faces A h / (|n| dim)."""
import itertools

import numpy as np


def _cell(i, pts, box, images, tol):
    dim = pts.shape[1]
    ri = pts[i]
    n_all, keys = [], []
    for s in images:
        x = pts + np.asarray(s) * box - ri
        for j in range(len(pts)):
            if j == i and not any(s):
                continue
            n_all.append(x[j])
            keys.append((j,) + tuple(int(v) for v in s))
    N = np.array(n_all)
    H = 0.5 * np.einsum("kd,kd->k", N, N)
    from scipy.spatial import HalfspaceIntersection
    A = np.hstack([N, -H[:, None]])                            # n.x - h <= 0
    hs = HalfspaceIntersection(A, np.zeros(dim))
    V = hs.intersections
    faces = {}
    vol = 0.0
    norms = np.linalg.norm(N, axis=1)
    ON = np.abs(V.dot(N.T) / norms - H / norms) <= tol          # [vertex, plane]: the vertex lies on the plane
    touching = np.nonzero(ON.sum(axis=0) >= dim)[0]
    for k in touching:
        n, h, key, nn = N[k], H[k], keys[k], norms[k]
        P = V[ON[:, k]]
        if dim == 2:
            if len(P) < 2:
                continue
            # the two extreme points along the edge direction
            t = np.array([-n[1], n[0]]) / nn
            u = P.dot(t)
            a, b = P[np.argmin(u)], P[np.argmax(u)]
            area = np.linalg.norm(b - a)
            cen = 0.5 * (a + b)
        else:
            if len(P) < 3:
                continue
            c0 = P.mean(axis=0)
            e1 = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 * nn else [0.0, 1.0, 0.0])
            e1 /= np.linalg.norm(e1)
            e2 = np.cross(n / nn, e1)
            ang = np.arctan2((P - c0).dot(e2), (P - c0).dot(e1))
            P = P[np.argsort(ang)]
            area, m = 0.0, np.zeros(3)
            for k in range(len(P)):
                a, b = P[k], P[(k + 1) % len(P)]
                at = 0.5 * np.cross(a - c0, b - c0).dot(n / nn)
                area += at
                m += at * (c0 + a + b) / 3.0
            cen = m / area if area != 0 else c0
            area = abs(area)
        vol += area * (h / nn) / dim
        faces[key] = (area, ri + cen)
    return faces, vol


def tessellate(points, box, area_tol=1e-12, vertex_tol=1e-10):
    """faces[i] = {(j, s_0, .., s_dim-1): (area, centroid)}, volumes [n]."""
    pts = np.asarray(points, np.float64)
    box = np.asarray(box, np.float64)
    n, dim = pts.shape
    h = (np.prod(box) / n) ** (1.0 / dim)
    images = list(itertools.product((-1, 0, 1), repeat=dim))
    faces, vols = [], np.empty(n)
    for i in range(n):
        f, v = _cell(i, pts, box, images, vertex_tol * h)
        faces.append({k: a for k, a in f.items() if a[0] > area_tol * h ** (dim - 1)})
        vols[i] = v
    return faces, vols


def face_list(faces, dim):
    """The faces listed once, as amm_create takes them: the side with the
    smaller cell index (or the positive image shift for a face with its own
    image); returns {(i, j, s..): (area, centroid)}."""
    out = {}
    for i, f in enumerate(faces):
        for key, val in f.items():
            j, s = key[0], key[1:]
            first_nonzero = next((v for v in s if v != 0), 0)
            if j > i or (j == i and first_nonzero > 0):
                out[(i,) + key] = val
    return out
