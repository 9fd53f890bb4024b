"""The two forms of the gradient estimate of Sec. 3.1, eq. (eqngrad2).

The paper writes V_i grad phi_i as the sum over the cell's faces of
A ([phi_j - phi_i] c / r + (phi_i + phi_j) n_out / 2), with c the face
centroid's offset from the midpoint of the two generators, r their distance
and n_out the outward unit normal.  A closed cell's vector area sum of
A n_out vanishes, so the estimate equals the sum of (phi_j - phi_i) w with
one weight w = A (c / r + n_out / 2) per face.  The GPU kernels use that
form, one weight per cell-face incidence.  These tests pin the reading:

- the cells the tessellator produces close to rounding (sum A n_out = 0);
- the oracle's unlimited gradients, which follow the paper's form, equal the
  sum of differences;
- on a uniform field the sum of differences is exactly zero, where the
  paper's form leaves phi times the rounding of the closure sum;
- where a cell does not close (one face's area altered by hand), the two
  forms differ by exactly phi_i sum A n_out / V (per face the paper's term
  exceeds the difference form's by A n_out ((phi_i + phi_j) - (phi_j -
  phi_i)) / 2 = A n_out phi_i), so the closure sum is the whole difference.
"""
import numpy as np
import pytest

from harness import ics
from harness.tess import tessellate
from oracle import oracle as O


def _mesh(dim, n, seed):
    rng = np.random.default_rng(seed)
    box = np.ones(dim)
    pts = ics.jittered_lattice((n,) * dim, box, 0.3, rng)
    return tessellate(pts, box)


def _faces(T):
    """Per face: left and right cells, unit normal L -> R, generator distance,
    centroid offset from the generators' midpoint, area."""
    L, R = T.cells[:, 0].astype(np.int64), T.cells[:, 1].astype(np.int64)
    rL = T.points[L]
    rR = T.points[R] + T.shift * T.box
    d = rR - rL
    r = np.linalg.norm(d, axis=1)
    n = d / r[:, None]
    c = T.centroid - 0.5 * (rL + rR)
    return L, R, n, r, c, T.area.astype(np.float64)


def _paper_form(T, phi, V, area=None):
    L, R, n, r, c, A = _faces(T)
    if area is not None:
        A = area
    g = np.zeros((T.n_cells, T.dim))
    # left cell: n_out = n; right cell: n_out = -n, the same c
    tL = A[:, None] * ((phi[R] - phi[L])[:, None] * c / r[:, None] + 0.5 * (phi[L] + phi[R])[:, None] * n)
    tR = A[:, None] * ((phi[L] - phi[R])[:, None] * c / r[:, None] - 0.5 * (phi[L] + phi[R])[:, None] * n)
    np.add.at(g, L, tL)
    np.add.at(g, R, tR)
    return g / V[:, None]


def _difference_form(T, phi, V, area=None):
    L, R, n, r, c, A = _faces(T)
    if area is not None:
        A = area
    g = np.zeros((T.n_cells, T.dim))
    wL = A[:, None] * (c / r[:, None] + 0.5 * n)       # weight of the left cell's incidence
    wR = A[:, None] * (c / r[:, None] - 0.5 * n)       # and of the right cell's
    np.add.at(g, L, (phi[R] - phi[L])[:, None] * wL)
    np.add.at(g, R, (phi[L] - phi[R])[:, None] * wR)
    return g / V[:, None]


def _closure(T, area=None):
    L, R, n, r, c, A = _faces(T)
    if area is not None:
        A = area
    s = np.zeros((T.n_cells, T.dim))
    np.add.at(s, L, A[:, None] * n)
    np.add.at(s, R, -A[:, None] * n)
    asum = np.bincount(L, weights=A, minlength=T.n_cells) + np.bincount(R, weights=A, minlength=T.n_cells)
    return s, asum


@pytest.mark.parametrize("dim,n,seed", [(3, 7, 3), (2, 13, 4)])
def test_cells_close(dim, n, seed):
    T = _mesh(dim, n, seed)
    s, asum = _closure(T)
    assert np.max(np.linalg.norm(s, axis=1) / asum) < 1e-12


@pytest.mark.parametrize("dim,n,seed", [(3, 7, 3), (2, 13, 4)])
def test_oracle_gradient_is_the_sum_of_differences(dim, n, seed):
    T = _mesh(dim, n, seed)
    M = O.Mesh(T)
    V, s = O.geometry(M)
    rng = np.random.default_rng(seed + 100)
    x = T.points
    W = np.zeros((T.n_cells, dim + 2))
    W[:, 0] = 1.0 + 0.3 * np.sin(2 * np.pi * x[:, 0]) + 0.05 * rng.standard_normal(T.n_cells)
    W[:, 1:dim + 1] = 0.5 * np.cos(2 * np.pi * x[:, :dim]) + 0.05 * rng.standard_normal((T.n_cells, dim))
    W[:, dim + 1] = 2.0 + 0.4 * np.cos(2 * np.pi * (x[:, 0] + x[:, 1]))
    g = O.gradients(M, W, V, s, limit=False)            # [n, dim + 2, dim]
    h = np.mean(V) ** (1.0 / dim)
    for a in range(dim + 2):
        gd = _difference_form(T, W[:, a], V)
        gp = _paper_form(T, W[:, a], V)
        scale = np.max(np.abs(W[:, a])) / h
        # the oracle follows the paper's form; the difference form agrees
        # to the rounding of the closure sums
        assert np.max(np.abs(g[:, a, :] - gp)) < 1e-12 * scale
        assert np.max(np.abs(g[:, a, :] - gd)) < 1e-11 * scale


@pytest.mark.parametrize("dim,n,seed", [(3, 7, 3), (2, 13, 4)])
def test_uniform_field_gives_zero_in_the_difference_form(dim, n, seed):
    T = _mesh(dim, n, seed)
    V, _ = O.geometry(O.Mesh(T))
    phi = np.full(T.n_cells, 1.2345e3)
    assert np.all(_difference_form(T, phi, V) == 0.0)
    # the paper's form leaves phi sum A n_out / V: rounding-sized, not zero
    gp = _paper_form(T, phi, V)
    h = np.mean(V) ** (1.0 / dim)
    assert np.max(np.abs(gp)) < 1e-10 * phi[0] / h


@pytest.mark.parametrize("dim,n,seed", [(3, 6, 5), (2, 11, 6)])
def test_unclosed_cell_differs_by_the_closure_term(dim, n, seed):
    T = _mesh(dim, n, seed)
    V, _ = O.geometry(O.Mesh(T))
    rng = np.random.default_rng(seed)
    phi = 1.0 + rng.random(T.n_cells)
    area = T.area.astype(np.float64).copy()
    area[0] *= 1.1                                       # face 0 no longer closes its two cells
    L0, R0 = int(T.cells[0, 0]), int(T.cells[0, 1])
    s, asum = _closure(T, area)
    assert np.linalg.norm(s[L0]) > 1e-3 * asum[L0]
    gp = _paper_form(T, phi, V, area)
    gd = _difference_form(T, phi, V, area)
    expect = phi[:, None] * s / V[:, None]
    h = np.mean(V) ** (1.0 / dim)
    assert np.max(np.abs((gp - gd) - expect)) < 1e-12 * np.max(phi) / h
    # only the two cells of the altered face differ beyond rounding
    big = np.linalg.norm(gp - gd, axis=1) > 1e-9 * np.max(phi) / h
    assert set(np.flatnonzero(big)) <= {L0, R0} and big[L0] and big[R0]
